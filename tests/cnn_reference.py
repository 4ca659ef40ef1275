"""FP32 PyTorch CPU reference of the learned pre-decoder network (test
infrastructure).  Parity unpinned against the paper: the network is not in
the paper; these functions only restate the network the C ABI documents, with
the same BF16 rounding points, so the CUDA kernels can be checked against it.

Rounding points mirrored from the kernels: weights of the three convolutions
are BF16; the outputs of the first two hidden layers are rounded to BF16; the
third layer's output and the head stay FP32."""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

C, IN_C = 16, 6
SIZES = [("w1", (C, IN_C, 3, 3, 3)), ("b1", (C,)), ("w2", (C, C, 3, 3, 3)), ("b2", (C,)),
         ("w3", (C, C, 3, 3, 3)), ("b3", (C,)), ("w4", (3, C)), ("b4", (3,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def random_params(seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    out = []
    for name, shape in SIZES:
        fan_in = int(np.prod(shape[1:])) if len(shape) > 1 else C
        scale = np.sqrt(2.0 / fan_in) if name.startswith("w") else 0.05
        out.append(rng.normal(0.0, scale, int(np.prod(shape))))
    return np.concatenate(out).astype(np.float32)


def unpack(params):
    p = torch.as_tensor(params, dtype=torch.float32)
    out, i = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[i:i + n].reshape(shape)
        i += n
    return out


def bf16(x):
    return x.to(torch.bfloat16).to(torch.float32)


def _ste_bf16(x):
    # rounds in the forward pass, identity in the backward pass
    return x + (bf16(x) - x).detach()


def features(L: int, s_prev: np.ndarray, s_cur: np.ndarray) -> torch.Tensor:
    """[S][3L^3] bits -> [S][6][L][L][L] (channels s_prev(n), s(n); site (z, y, x))."""
    S = s_prev.shape[0]
    a = s_prev.reshape(S, 3, L, L, L).astype(np.float32)
    b = s_cur.reshape(S, 3, L, L, L).astype(np.float32)
    return torch.from_numpy(np.concatenate([a, b], axis=1))


def _conv(x, w):
    return F.conv3d(F.pad(x, (1, 1, 1, 1, 1, 1), mode="circular"), w)


def logits(params, L, s_prev, s_cur, train=False):
    """[S][3][L^3] logits; with train=True the rounding is straight-through."""
    P = unpack(params)
    rnd = _ste_bf16 if train else bf16
    x = features(L, s_prev, s_cur)
    h1 = rnd(torch.relu(_conv(x, bf16(P["w1"])) + P["b1"].view(1, -1, 1, 1, 1)))
    h2 = rnd(torch.relu(_conv(h1, bf16(P["w2"])) + P["b2"].view(1, -1, 1, 1, 1)))
    h3 = torch.relu(_conv(h2, bf16(P["w3"])) + P["b3"].view(1, -1, 1, 1, 1))
    z = torch.einsum("scxyz,dc->sdxyz", h3, P["w4"]) + P["b4"].view(1, -1, 1, 1, 1)
    return z.reshape(z.shape[0], 3, -1)


def loss_and_grad(params, L, s_prev, s_cur, labels):
    """Summed BCE over all edges and samples, and the gradient of the mean BCE
    (the quantity the training step minimises) with respect to the FP32
    master parameters.  labels: [S][3L^3] bits."""
    p = torch.tensor(params, dtype=torch.float32, requires_grad=True)
    z = logits(p, L, s_prev, s_cur, train=True)
    y = torch.from_numpy(labels.reshape(z.shape).astype(np.float32))
    per = F.binary_cross_entropy_with_logits(z, y, reduction="none")
    mean = per.mean()
    mean.backward()
    return float(per.sum()), p.grad.numpy().copy()
