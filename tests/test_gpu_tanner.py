"""The decoders on generic Tanner graphs (the question of Sec. 5) against the
oracle, through the C ABI: noise, measurement and flip / p-flip schedules
bit-exact; BP message by message (per-iteration protocol, as for the toric
BP) and by its decisions.  Codes: the 3D toric code's own graph (where the
generic calls must equal the toric ones), a hypergraph product of two
(3,4)-biregular classical codes, and a random code with check degrees up to
32 (the degree-specialised and looped check nodes, the 6-bit counters)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2212_06985_gb300 as t3d
import toric3d_inputs as inp
from gpu_util import dev, download_bits, upload_bits, workspace

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _random_code(n, m, seed):
    """Checks of degree 2..12, two of degree 20 and 32, variable 0 in 32 checks; no
    repeated variable."""
    rng = np.random.default_rng(seed)
    degs = rng.integers(2, 13, m)
    degs[:2] = [20, 32]
    rows = [rng.choice(n, int(d), replace=False) for d in degs]
    for c in range(m):
        if c < 32 and 0 not in rows[c]:
            rows[c][-1] = 0
        elif c >= 32 and 0 in rows[c]:
            free = np.setdiff1d(np.arange(1, n), rows[c])
            rows[c][rows[c] == 0] = free[0]
    return inp.csr([np.sort(r) for r in rows])


def _codes():
    cptr, cvar, n = inp.hgp_workload(16, 5)
    yield "hgp16", cptr, cvar, n
    cptr, cvar = _random_code(120, 90, 2)
    yield "random", cptr, cvar, 120
    cptr, cvar = oracle.toric_tanner(3)
    yield "toric3", cptr, cvar, 81


CODES = {name: (cptr, cvar, n) for name, cptr, cvar, n in _codes()}


def _graph(name):
    cptr, cvar, n = CODES[name]
    return cptr, cvar, n, t3d.tanner_prepare(cptr, cvar, n)


def test_prepare_describes_the_graph():
    cptr, cvar, n, g = _graph("random")
    assert g.n_vars == n and g.n_checks == len(cptr) - 1 and g.n_edges == len(cvar)
    assert g.desc.max_check_degree == 32
    assert g.desc.max_var_degree == int(np.bincount(cvar).max()) == 32


def test_prepare_rejects_bad_lists():
    blob = workspace(1 << 16)
    desc = t3d.Tanner()
    import ctypes

    def prep(cptr, cvar, n):
        cptr = np.asarray(cptr, np.int32)
        cvar = np.asarray(cvar, np.int32)
        return t3d.lib().toric3d_tanner_prepare(n, len(cptr) - 1, cptr.ctypes.data_as(ctypes.c_void_p),
                                                cvar.ctypes.data_as(ctypes.c_void_p),
                                                ctypes.c_void_p(blob.data_ptr()), blob.numel(), ctypes.byref(desc))
    assert prep([0, 2, 4], [0, 1, 1, 2], 3) == 0
    assert prep([0, 2, 4], [0, 0, 1, 2], 3) != 0            # variable twice in a check
    assert prep([0, 2, 4], [0, 3, 1, 2], 3) != 0            # out of range
    assert prep([0, 33], list(range(33)), 40) != 0          # check degree 33
    assert prep([1, 2], [0, 1], 3) != 0                     # cptr[0] != 0


def test_toric_graph_equals_toric_calls():
    """On the toric code's own graph the generic noise, measurement and flip equal the toric calls."""
    L, S = 4, 200
    n = 3 * L ** 3
    cptr, cvar = oracle.toric_tanner(L)
    g = t3d.tanner_prepare(cptr, cvar, n)
    W = inp.words_for(S)
    z = lambda: torch.zeros((n, W), dtype=torch.int64, device=dev())
    e1, s1, e2, s2 = z(), z(), z(), z()
    t3d.toric3d_tanner_noise(g, S, e1, 0.06, 5, 128, 2)
    t3d.toric3d_noise(L, e2, 0.06, 5, 128, 2)
    t3d.toric3d_tanner_syndrome(g, S, e1, s1, 0.04, 5, 128, 2)
    t3d.toric3d_syndrome(L, e2, s2, 0.04, 5, 128, 2)
    torch.cuda.synchronize()
    assert torch.equal(e1, e2) and torch.equal(s1, s2)
    t3d.toric3d_tanner_pflip(g, S, e1, s1, "F", 3, 0, 5, 128, 2, workspace(t3d.toric3d_tanner_flip_workspace_bytes(g, S)))
    t3d.toric3d_flip(L, e2, s2, 3, workspace(t3d.toric3d_flip_workspace_bytes(L, W)))
    torch.cuda.synchronize()
    assert torch.equal(e1, e2) and torch.equal(s1, s2)


@pytest.mark.parametrize("name,S,sample0", [("hgp16", 200, 64), ("random", 64 * 3 + 7, 0), ("toric3", 65, 128)])
def test_noise_measure_schedule_bit_exact(name, S, sample0):
    cptr, cvar, n, g = _graph(name)
    m = len(cptr) - 1
    W = inp.words_for(S)
    e = torch.zeros((n, W), dtype=torch.int64, device=dev())
    s = torch.zeros((m, W), dtype=torch.int64, device=dev())
    work = workspace(t3d.toric3d_tanner_flip_workspace_bytes(g, S))
    ora_e = np.zeros((S, n), np.uint8)
    seed, sched = 13, "PFFPFFP"
    for cycle in (1, 2):
        t3d.toric3d_tanner_noise(g, S, e, 0.05, seed, sample0, cycle)
        t3d.toric3d_tanner_syndrome(g, S, e, s, 0.03, seed, sample0, cycle)
        ora_e = oracle.tanner_noise_batch(ora_e, 0.05, seed, sample0, cycle)
        ora_s = oracle.tanner_measure_batch(cptr, cvar, ora_e, 0.03, seed, sample0, cycle)
        torch.cuda.synchronize()
        assert np.array_equal(download_bits(e, S), ora_e) and np.array_equal(download_bits(s, S), ora_s)
        t3d.toric3d_tanner_pflip(g, S, e, s, sched, 9, 4, seed, sample0, cycle, work)
        for k in range(9):
            ora_e, ora_s = oracle.tanner_rule_batch(cptr, cvar, ora_e, ora_s, sched[k % len(sched)] == "P", seed,
                                                    sample0, cycle, 4 + k)
        torch.cuda.synchronize()
        assert np.array_equal(download_bits(e, S), ora_e) and np.array_equal(download_bits(s, S), ora_s)


def test_logical_parities_through_a_logical_graph():
    """Logical readout of a generic code: the syndrome of e with respect to a graph whose
    rows are qubit sets (here straight lines of the hypergraph product of two cycles, the
    2D toric code) is the parity of e on each set, bit-exact; with logical operators as
    the rows this is the readout."""
    L, S = 6, 150
    X, Z, n = inp.hypergraph_product(inp.cyclic_repetition(L), L, inp.cyclic_repetition(L), L)
    # qubits (a, b) -> a L + b: the line a = 0 and the line b = 0 of the first block, and the
    # same two lines of the second block (n1 n2 + i L + j)
    logicals = [[b for b in range(L)], [a * L for a in range(L)],
                [L * L + j for j in range(L)], [L * L + i * L for i in range(L)]]
    lptr, lvar = inp.csr(logicals)
    g = t3d.tanner_prepare(lptr, lvar, n)
    ebits = inp.random_bits(S, n, 0.2, 3)
    e = upload_bits(ebits)
    out = torch.zeros((len(logicals), inp.words_for(S)), dtype=torch.int64, device=dev())
    t3d.toric3d_tanner_syndrome(g, S, e, out, 0.0, 1, 0, 1)
    torch.cuda.synchronize()
    want = np.stack([ebits[:, l].sum(axis=1) % 2 for l in logicals], axis=1).astype(np.uint8)
    assert np.array_equal(download_bits(out, S), want)


def _rows_bound(cptr, cvar, prior, cv_in, n):
    """Per Tanner edge: the FP32 rounding of the other inputs of its check (each input
    T_v - M is a sum of deg_v + 2 terms: (deg_v + 2) u times the magnitudes)."""
    A = np.zeros(n)
    np.add.at(A, cvar, np.abs(cv_in))
    deg = np.bincount(cvar, minlength=n)
    xb = (deg + 2) * U32 * (np.abs(prior) + A)
    per_check = np.add.reduceat(xb[cvar], cptr[:-1])
    return np.repeat(per_check, np.diff(cptr)) - xb[cvar]


@pytest.mark.parametrize("name,S,iters", [("hgp16", 70, 6), ("random", 64, 6), ("toric3", 33, 5)])
def test_bp_each_iteration_matches_oracle(name, S, iters):
    cptr, cvar, n, g = _graph(name)
    m = len(cptr) - 1
    rng = np.random.default_rng(7)
    prior32 = rng.uniform(1.5, 4.0, n).astype(np.float32)        # per-variable priors
    prior = prior32.astype(np.float64)
    ebits = inp.random_bits(S, n, 0.06, 8)
    sbits = oracle.tanner_syndrome_batch(cptr, cvar, ebits) ^ inp.random_bits(S, m, 0.03, 9)
    s = upload_bits(sbits)
    mb = t3d.toric3d_tanner_bp_message_bytes(g, S)
    Sp = 64 * inp.words_for(S)
    cur = torch.zeros(mb // 4, dtype=torch.float32, device=dev())
    nxt = torch.zeros_like(cur)
    work = workspace(n * Sp * 4)
    pr = torch.from_numpy(prior32).to(dev())
    worst = 0.0
    for it in range(iters):
        t3d.toric3d_tanner_bp_step(g, S, s, pr, cur, nxt, work)
        torch.cuda.synchronize()
        m_in = cur.cpu().numpy().astype(np.float64).reshape(len(cvar), Sp)
        m_out = nxt.cpu().numpy().astype(np.float64).reshape(len(cvar), Sp)
        for i in range(S):
            _, ref = oracle.bp_priors_from(cptr, cvar, sbits[i], prior, 1, m_in[:, i])
            tol = (1e-5 * np.abs(ref) + 1e-6 + 2.3e-16 * np.exp(np.minimum(np.abs(ref), 40.0))
                   + _rows_bound(cptr, cvar, prior, m_in[:, i], n))
            err = np.abs(m_out[:, i] - ref)
            assert (err <= tol).all(), (it, i, float(err.max()))
            worst = max(worst, float((err / tol).max()))
        cur, nxt = nxt, cur
    print(f"{name}: worst error / tolerance over {iters} iterations: {worst:.3f}")


@pytest.mark.parametrize("name,S,iters,chunk", [("hgp16", 150, 8, None), ("random", 130, 10, 64),
                                                ("toric3", 64, 12, None)])
def test_bp_decisions_match_oracle(name, S, iters, chunk):
    cptr, cvar, n, g = _graph(name)
    m = len(cptr) - 1
    prior32 = np.full(n, np.log(0.95 / 0.05), dtype=np.float32)
    ebits = inp.random_bits(S, n, 0.05, 3)
    sbits = oracle.tanner_syndrome_batch(cptr, cvar, ebits)
    e, s = upload_bits(ebits), upload_bits(sbits)
    llr = None if chunk else torch.zeros((n, S), dtype=torch.float32, device=dev())
    work = workspace(t3d.toric3d_tanner_bp_workspace_bytes(g, chunk or S))
    t3d.toric3d_tanner_bp(g, S, e, s, torch.from_numpy(prior32).to(dev()), iters, work, llr)
    torch.cuda.synchronize()
    e_ref, s_ref, ref = oracle.tanner_bp_batch(cptr, cvar, ebits, sbits, prior32.astype(np.float64), iters)
    got_e, got_s = download_bits(e, S), download_bits(s, S)
    rows = (np.abs(ref) > 1e-3).all(axis=1)
    assert rows.mean() > 0.8
    assert np.array_equal(got_e[rows], e_ref[rows]) and np.array_equal(got_s[rows], s_ref[rows])
    # every sample: the update is a decision d applied as e ^= d, s ^= H d
    d = got_e ^ ebits
    assert np.array_equal(got_s ^ sbits, oracle.tanner_syndrome_batch(cptr, cvar, d))
    if llr is not None:
        g_llr = llr.cpu().numpy().T
        assert np.array_equal(d, (g_llr < 0).astype(np.uint8))
        clear = np.abs(ref) > 1e-3
        assert np.array_equal((g_llr < 0)[clear], (ref < 0)[clear])


def test_bp_chunking_is_invisible():
    cptr, cvar, n, g = _graph("hgp16")
    S = 64 * 3 + 5
    prior = torch.full((n,), 3.0, dtype=torch.float32, device=dev())
    ebits = inp.random_bits(S, n, 0.05, 4)
    sbits = oracle.tanner_syndrome_batch(cptr, cvar, ebits)
    outs = []
    for chunk in (64, 128, S):
        e, s = upload_bits(ebits), upload_bits(sbits)
        t3d.toric3d_tanner_bp(g, S, e, s, prior, 9, workspace(t3d.toric3d_tanner_bp_workspace_bytes(g, chunk)))
        torch.cuda.synchronize()
        outs.append((download_bits(e, S), download_bits(s, S)))
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1])


def test_hgp_full_size_sampled():
    """The hypergraph-product workload at full size (250,000 qubits, 120,000 checks):
    one noisy cycle, BP and a p-flip schedule, sampled samples against the oracle."""
    cptr, cvar, n = inp.hgp_workload(400, 1)
    m = len(cptr) - 1
    g = t3d.tanner_prepare(cptr, cvar, n)
    S, seed = 256, 3
    W = inp.words_for(S)
    e = torch.zeros((n, W), dtype=torch.int64, device=dev())
    s = torch.zeros((m, W), dtype=torch.int64, device=dev())
    t3d.toric3d_tanner_noise(g, S, e, 0.03, seed, 0, 1)
    t3d.toric3d_tanner_syndrome(g, S, e, s, 0.03, seed, 0, 1)
    prior = torch.full((n,), float(np.log(0.97 / 0.03)), dtype=torch.float32, device=dev())
    e_bp = e.clone()
    s_bp = s.clone()
    t3d.toric3d_tanner_bp(g, S, e_bp, s_bp, prior, 10, workspace(t3d.toric3d_tanner_bp_workspace_bytes(g, S)))
    t3d.toric3d_tanner_pflip(g, S, e, s, "PFF", 3, 0, seed, 0, 1, workspace(t3d.toric3d_tanner_flip_workspace_bytes(g, S)))
    torch.cuda.synchronize()
    pick = [0, 63, 64, 255]
    e0 = np.stack([oracle.tanner_noise_batch(np.zeros((1, n), np.uint8), 0.03, seed, i, 1)[0] for i in pick])
    s0 = np.stack([oracle.tanner_measure_batch(cptr, cvar, e0[k:k + 1], 0.03, seed, pick[k], 1)[0]
                   for k in range(len(pick))])
    ef, sf = e0.copy(), s0.copy()
    for k, kind in enumerate("PFF"):
        for j, i in enumerate(pick):
            a, b = oracle.tanner_rule_batch(cptr, cvar, ef[j:j + 1], sf[j:j + 1], kind == "P", seed, i, 1, k)
            ef[j], sf[j] = a[0], b[0]
    got_e, got_s = download_bits(e, S), download_bits(s, S)
    assert np.array_equal(got_e[pick], ef) and np.array_equal(got_s[pick], sf)
    e_ref, s_ref, ref = oracle.tanner_bp_batch(cptr, cvar, e0, s0, np.full(n, np.log(0.97 / 0.03)), 10)
    got_e, got_s = download_bits(e_bp, S), download_bits(s_bp, S)
    for j, i in enumerate(pick):
        if (np.abs(ref[j]) > 1e-3).all():
            assert np.array_equal(got_e[i], e_ref[j]) and np.array_equal(got_s[i], s_ref[j]), i
