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


@pytest.mark.parametrize("L,S", [(4, 64), (5, 200), (3, 300)])
def test_cnn_gradient_matches_reference(L, S):
    # 200 and 300 samples: two and three 128-sample tiles, the last one partly padding
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


def _patch_logits(params, L, sp_bits, sc_bits, site):
    """Reference logits of one site from its 7x7x7 periodic neighbourhood (three valid
    3x3x3 convolutions shrink 7 -> 5 -> 3 -> 1)."""
    import torch.nn.functional as F
    P = ref.unpack(params)
    L3 = L ** 3
    z0, y0, x0 = site // (L * L), (site // L) % L, site % L
    idx = np.array([[[((z % L) * L + (y % L)) * L + (x % L) for x in range(x0 - 3, x0 + 4)]
                     for y in range(y0 - 3, y0 + 4)] for z in range(z0 - 3, z0 + 4)])
    feat = np.stack([sp_bits[c * L3 + idx] for c in range(3)] + [sc_bits[c * L3 + idx] for c in range(3)])
    x = torch.from_numpy(feat[None].astype(np.float32))
    h = ref.bf16(torch.relu(F.conv3d(x, ref.bf16(P["w1"])) + P["b1"].view(1, -1, 1, 1, 1)))
    h = ref.bf16(torch.relu(F.conv3d(h, ref.bf16(P["w2"])) + P["b2"].view(1, -1, 1, 1, 1)))
    h = torch.relu(F.conv3d(h, ref.bf16(P["w3"])) + P["b3"].view(1, -1, 1, 1, 1))
    return (P["w4"] @ h[0, :, 0, 0, 0] + P["b4"]).numpy()


def test_cnn_full_size_sampled_decisions():
    """L = 32 with a 16,384-sample launch (the bench's pre-decoder chunk): the decisions the
    kernels apply to e at 300 sampled (site, sample) pairs equal the reference's sign wherever
    |logit| > 0.05."""
    from paper_2212_06985_gb300 import learned
    L, S = 32, 16384
    n, W = 3 * L ** 3, inp.words_for(S)
    params = learned.load_params(learned.__file__.replace("learned.py", "weights/cnn_L12_p04.npz"))
    g = torch.Generator(device=dev())
    g.manual_seed(3)
    rnd = lambda: torch.randint(-2 ** 62, 2 ** 62, (n, W), dtype=torch.int64, device=dev(), generator=g)
    sp = rnd() & rnd() & rnd()           # about 1/8 of the checks unsatisfied
    sc = sp ^ (rnd() & rnd() & rnd() & rnd())
    e = torch.zeros_like(sp)
    _, blob = _blob(params)
    t3d.toric3d_cnn_decode(L, S, sp, sc.clone(), e, blob, workspace(t3d.toric3d_cnn_workspace_bytes(L, S)))
    torch.cuda.synchronize()
    t3d.toric3d_cnn_status()
    rng = np.random.default_rng(4)
    samples = rng.integers(0, S, 30)
    sites = rng.integers(0, L ** 3, 10)
    ew, spw, scw = (t.cpu().numpy().view(np.uint64) for t in (e, sp, sc))
    checked = 0
    for j in samples:
        bit = lambda words: ((words[:, j // 64] >> np.uint64(j % 64)) & np.uint64(1)).astype(np.uint8)
        spb, scb, eb = bit(spw), bit(scw), bit(ew)
        for r in sites:
            z = _patch_logits(params, L, spb, scb, int(r))
            for d in range(3):
                if abs(z[d]) > 0.05:
                    assert eb[d * L ** 3 + r] == int(z[d] > 0), (j, r, d, z[d])
                    checked += 1
    assert checked > 600


def test_cnn_bounded_wait_gives_up_and_the_context_stays_usable():
    """A 1 ns bound makes the tensor-core kernels' waits run out (nothing faults:
    the wind-down still drains the kernel's own copies and MMAs for up to 1 s and
    frees its TMEM).  The status call reports T3D_ETIMEOUT once; with the bound
    restored the same decode on the same context matches the reference."""
    L, S = 4, 96
    n = 3 * L ** 3
    params = ref.random_params(L)
    sp = inp.random_bits(S, n, 0.15, 10 + L)
    sc = inp.random_bits(S, n, 0.15, 20 + L)
    _, blob = _blob(params)
    work = workspace(t3d.toric3d_cnn_workspace_bytes(L, S))
    logits = torch.zeros((3, L ** 3, S), dtype=torch.float32, device=dev())
    t3d.toric3d_cnn_status()                                   # start from a clear flag
    t3d.toric3d_cnn_debug_wait_limit(1)
    try:
        t3d.toric3d_cnn_decode(L, S, upload_bits(sp), upload_bits(sc), upload_bits(np.zeros_like(sc)), blob, work,
                               logits)
        with pytest.raises(t3d.T3DError) as exc:
            t3d.toric3d_cnn_status()
        assert exc.value.status == 3                           # T3D_ETIMEOUT
        t3d.toric3d_cnn_status()                               # the flag was cleared by the read
    finally:
        t3d.toric3d_cnn_debug_wait_limit(0)
    with pytest.raises(t3d.T3DError):
        t3d.toric3d_cnn_debug_wait_limit(2_000_000_000)        # above the 1 s maximum
    e = upload_bits(np.zeros_like(sc))
    t3d.toric3d_cnn_decode(L, S, upload_bits(sp), upload_bits(sc), e, blob, work, logits)
    torch.cuda.synchronize()
    t3d.toric3d_cnn_status()
    g = logits.cpu().numpy().transpose(2, 0, 1).reshape(S, 3, -1)
    z = ref.logits(params, L, sp, sc).numpy()
    assert np.abs(g - z).max() < 0.02 + 0.01 * np.abs(z).max()
