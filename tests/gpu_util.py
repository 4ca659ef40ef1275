"""Test glue between the oracle's [sample][bit] uint8 arrays and the library's
bit-sliced device tensors, plus the documented BP message layout."""
from __future__ import annotations

import numpy as np
import torch

import toric3d_inputs as inp


def dev():
    return torch.device("cuda:0")


def upload_bits(bits: np.ndarray) -> torch.Tensor:
    """[S][n] uint8 -> device int64 [n][W] (bit-sliced)."""
    return torch.from_numpy(inp.pack(bits).view(np.int64)).to(dev())


def download_bits(words: torch.Tensor, n_samples: int) -> np.ndarray:
    return inp.unpack(words.cpu().numpy().view(np.uint64), n_samples)


def zeros_words(n: int, S: int) -> torch.Tensor:
    return torch.zeros((n, inp.words_for(S)), dtype=torch.int64, device=dev())


def workspace(nbytes: int) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=dev())


def message_index(L: int, face_edges) -> np.ndarray:
    """For every oracle Tanner edge 4f + j (face f -> its j-th edge in the
    oracle's face order), the flat offset within one 64-sample word row of the
    library's message buffer float[words][L^3][3][4][64] (sample 0 of the row)."""
    L3 = L ** 3
    n = 3 * L3
    out = np.zeros(4 * n, dtype=np.int64)
    for f in range(n):
        normal = f // L3
        a, b = [x for x in range(3) if x != normal]
        slots = [2 * (b - 1), 2 * (b - 1) + 1, 2 * a, 2 * a + 1]
        for j in range(4):
            v = int(face_edges[f][j])
            d, site = v // L3, v % L3
            out[4 * f + j] = ((site * 3 + d) * 4 + slots[j]) * 64
    return out


def gpu_messages_to_oracle(msg: torch.Tensor, L: int, n_samples: int, idx: np.ndarray) -> np.ndarray:
    """Library message buffer -> [S][4*3L^3] float64 in oracle Tanner-edge order."""
    per_word = 3 * L ** 3 * 4 * 64
    m = msg.detach().cpu().numpy().astype(np.float64).reshape(-1, per_word)
    out = np.empty((n_samples, len(idx)))
    for s in range(n_samples):
        out[s] = m[s // 64, idx + (s % 64)]
    return out
