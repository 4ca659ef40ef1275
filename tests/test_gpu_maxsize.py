"""The largest lattices the calls accept, checked through properties that hold
at any size (an oracle run per sample would take minutes there): L = 256 for
the bit-sliced calls (noise, syndrome, flip, p-flip, logical readout) and
L = 128 for BP.  Isolated errors, some on the periodic boundary, light exactly
the four faces that contain them (Sec. 2) and are removed by one flip or
p-flip application (Sec. 3.1: a lone error has all four checks unsatisfied,
its neighbours one); BP corrects them too (Sec. 4.1)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2212_06985_gb300 as t3d
from gpu_util import dev, workspace

pytestmark = pytest.mark.gpu


def _edge(L, d, x, y, z):
    return ((d * L + z) * L + y) * L + x


def _isolated(L):
    """One edge per sample (64 samples): the corners and faces of the periodic box."""
    coords = [(0, 0, 0), (L - 1, L - 1, L - 1), (L - 1, 0, 0), (0, L - 1, 0), (0, 0, L - 1), (L // 2, L // 3, 7)]
    edges = [_edge(L, d, *c) for c in coords for d in range(3)]
    return (edges * 4)[:64]


def _state(L, edges):
    """Bit-sliced error state with edge edges[i] set in sample i (64 samples, one word)."""
    n = 3 * L ** 3
    e = torch.zeros((n, 1), dtype=torch.int64, device=dev())
    words = {}
    for i, v in enumerate(edges):
        words[v] = words.get(v, 0) | (1 << i)
    idx = torch.tensor(list(words.keys()), dtype=torch.int64, device=dev())
    val = torch.tensor([w - (1 << 64) if w >= (1 << 63) else w for w in words.values()], dtype=torch.int64,
                       device=dev())
    e[idx, 0] = val
    return e


def _faces_of(L, v):
    """The four faces containing edge v: for each normal n != d (c the third axis), the
    faces (n, r) and (n, r - e_c); each checked against the oracle's face -> edge map."""
    L3 = L ** 3
    d, site = divmod(v, L3)
    r = [site % L, (site // L) % L, site // (L * L)]
    out = []
    for n in range(3):
        if n == d:
            continue
        c = 3 - d - n
        for shift in (0, -1):
            q = list(r)
            q[c] = (q[c] + shift) % L
            f = n * L3 + (q[2] * L + q[1]) * L + q[0]
            assert v in oracle.face_edges(L, f)
            out.append(f)
    return sorted(out)


@pytest.mark.parametrize("rule", ["F", "P"])
def test_L256_single_errors(rule):
    L = 256
    edges = _isolated(L)
    e = _state(L, edges)
    s = torch.zeros_like(e)
    t3d.toric3d_syndrome(L, e, s, 0.0, 1, 0, 1)
    torch.cuda.synchronize()
    nz = torch.nonzero(s[:, 0]).flatten()
    assert len(nz) <= 4 * len(set(edges))
    rows = s[nz, 0].cpu().numpy().view(np.uint64)
    for i, v in enumerate(edges[:18]):
        lit = sorted(int(f) for f, wv in zip(nz.cpu().numpy(), rows) if (int(wv) >> i) & 1)
        assert lit == _faces_of(L, v), (i, v)
    work = workspace(t3d.toric3d_flip_workspace_bytes(L, 1))
    t3d.toric3d_pflip(L, e, s, rule, 1, 0, 3, 0, 1, work)
    torch.cuda.synchronize()
    assert not torch.any(e) and not torch.any(s)
    mask = torch.zeros(64, dtype=torch.uint8, device=dev())
    t3d.toric3d_logical(L, 64, e, mask)
    torch.cuda.synchronize()
    assert not torch.any(mask)


def test_L256_noise_rate_and_logical_of_a_line():
    """Noise at p = 1/16 over 50M edges x 64 samples hits its rate; a full straight
    line of x-edges is one odd line of L^2, far from a majority: no logical failure."""
    L = 256
    n = 3 * L ** 3
    e = torch.zeros((n, 1), dtype=torch.int64, device=dev())
    t3d.toric3d_noise(L, e, 1 / 16, 5, 0, 1)
    torch.cuda.synchronize()
    ones = int(sum(bin(int(x) & ((1 << 64) - 1)).count("1") for x in e[::4099, 0].cpu().numpy()))
    seen = 64 * len(range(0, n, 4099))
    assert abs(ones / seen - 1 / 16) < 0.004
    line = torch.zeros_like(e)
    line[[_edge(L, 0, x, 5, 9) for x in range(L)], 0] = 1
    mask = torch.zeros(64, dtype=torch.uint8, device=dev())
    t3d.toric3d_logical(L, 64, line, mask)
    torch.cuda.synchronize()
    assert not torch.any(mask)


def test_L128_bp_corrects_single_errors():
    L = 128
    edges = _isolated(L)
    e = _state(L, edges)
    s = torch.zeros_like(e)
    t3d.toric3d_syndrome(L, e, s, 0.0, 1, 0, 1)
    work = workspace(t3d.toric3d_bp_workspace_bytes(L, 64))
    t3d.toric3d_bp(L, 64, e, s, 0.01, 0.01, 10, work)
    torch.cuda.synchronize()
    assert not torch.any(e) and not torch.any(s)
