"""The pre-decoder's CUDA kernels against the FP32 PyTorch CPU reference of the
same network (cnn_reference.py; parity unpinned against the paper, which has
no such network): logits and the corrections they apply, the gradient of a
training step, and Adam decreasing the loss."""
import numpy as np
import pytest
import torch

import cnn_reference as ref
import oracle
import paper_2212_06985_gb300 as t3d
import toric3d_inputs as inp
from gpu_util import dev, download_bits, upload_bits, workspace

pytestmark = pytest.mark.gpu


def _blob(params):
    p = torch.from_numpy(params).to(dev())
    blob = workspace(t3d.toric3d_cnn_blob_bytes())
    t3d.toric3d_cnn_prepare(p, blob)
    return p, blob


@pytest.mark.parametrize("L,S", [(4, 96), (5, 64), (3, 200), (8, 300), (12, 130), (2, 70)])
def test_cnn_logits_and_corrections_match_reference(L, S):
    n = 3 * L ** 3
    params = ref.random_params(L)
    sp = inp.random_bits(S, n, 0.15, 10 + L)
    sc = inp.random_bits(S, n, 0.15, 20 + L)
    e0 = inp.random_bits(S, n, 0.05, 30 + L)
    _, blob = _blob(params)
    e, s, s_prev = upload_bits(e0), upload_bits(sc), upload_bits(sp)
    logits = torch.zeros((3, L ** 3, S), dtype=torch.float32, device=dev())
    t3d.toric3d_cnn_decode(L, S, s_prev, s, e, blob, workspace(t3d.toric3d_cnn_workspace_bytes(L, S)), logits)
    torch.cuda.synchronize()
    t3d.toric3d_cnn_status()
    g = logits.cpu().numpy().transpose(2, 0, 1).reshape(S, 3, -1)
    z = ref.logits(params, L, sp, sc).numpy()
    err = np.abs(g - z)
    print(f"max |logit error| {err.max():.3e}, max |logit| {np.abs(z).max():.2f}")
    assert err.max() < 0.02 + 0.01 * np.abs(z).max()
    clear = np.abs(z) > 0.05
    assert np.array_equal((g > 0)[clear], (z > 0)[clear])
    d = (g > 0).reshape(S, n).astype(np.uint8)
    assert np.array_equal(download_bits(e, S), e0 ^ d)
    assert np.array_equal(download_bits(s, S), sc ^ oracle.syndrome_batch(L, d))


def test_cnn_gradient_matches_reference():
    L, S = 4, 64
    n = 3 * L ** 3
    params = ref.random_params(7)
    sp = inp.random_bits(S, n, 0.15, 1)
    sc = inp.random_bits(S, n, 0.15, 2)
    y = inp.random_bits(S, n, 0.08, 3)
    p, blob = _blob(params)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    grads = torch.zeros_like(p)
    loss = torch.zeros(1, dtype=torch.float32, device=dev())
    work = workspace(t3d.toric3d_cnn_train_workspace_bytes(L, S))
    t3d.toric3d_cnn_train_step(L, S, upload_bits(sp), upload_bits(sc), upload_bits(y), p, m, v, 1, 0.0,
                               blob, work, loss, grads_out=grads)
    torch.cuda.synchronize()
    ref_loss, ref_g = ref.loss_and_grad(params, L, sp, sc, y)
    gg = grads.cpu().numpy()
    assert abs(float(loss.item()) - ref_loss) < 2e-3 * ref_loss
    cos = float(np.dot(gg, ref_g) / (np.linalg.norm(gg) * np.linalg.norm(ref_g)))
    rel = float(np.abs(gg - ref_g).max() / np.abs(ref_g).max())
    print(f"gradient cosine {cos:.6f}, max error / max |g| {rel:.3e}")
    assert cos > 0.999 and rel < 0.05
    assert np.array_equal(p.cpu().numpy(), params)          # lr = 0 leaves the parameters


def test_cnn_adam_steps_reduce_the_loss():
    L, S = 4, 128
    n = 3 * L ** 3
    params = ref.random_params(9)
    sp = inp.random_bits(S, n, 0.1, 4)
    sc = inp.random_bits(S, n, 0.1, 5)
    y = inp.random_bits(S, n, 0.05, 6)
    p, blob = _blob(params)
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    loss = torch.zeros(1, dtype=torch.float32, device=dev())
    work = workspace(t3d.toric3d_cnn_train_workspace_bytes(L, S))
    args = (upload_bits(sp), upload_bits(sc), upload_bits(y))
    losses = []
    for step in range(1, 41):
        t3d.toric3d_cnn_train_step(L, S, *args, p, m, v, step, 3e-3, blob, work, loss)
        losses.append(float(loss.item()))
    assert losses[-1] < 0.7 * losses[0]
