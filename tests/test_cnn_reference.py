"""CPU checks of the pre-decoder's PyTorch reference and host helpers: the
parameter count the ABI documents, the circular-padding convention (a shifted
input shifts the output), and that its gradient matches finite differences."""
import numpy as np
import torch

import cnn_reference as ref
import paper_2212_06985_gb300 as t3d
import toric3d_inputs as inp


def test_param_count_matches_library():
    assert ref.N_PARAMS == 16515 == t3d.toric3d_cnn_param_count()


def test_translation_equivariance():
    L = 4
    params = ref.random_params(1)
    sp = inp.random_bits(2, 3 * L ** 3, 0.2, 1)
    sc = inp.random_bits(2, 3 * L ** 3, 0.2, 2)
    z = ref.logits(params, L, sp, sc).reshape(2, 3, L, L, L)
    roll = lambda a: np.roll(a.reshape(2, 3, L, L, L), 1, axis=4).reshape(2, -1)
    z2 = ref.logits(params, L, roll(sp), roll(sc)).reshape(2, 3, L, L, L)
    assert torch.allclose(torch.roll(z, 1, dims=4), z2, atol=1e-5)


def test_gradient_matches_finite_differences():
    L = 3
    params = ref.random_params(3).astype(np.float64).astype(np.float32)
    sp = inp.random_bits(2, 3 * L ** 3, 0.2, 4)
    sc = inp.random_bits(2, 3 * L ** 3, 0.2, 5)
    y = inp.random_bits(2, 3 * L ** 3, 0.1, 6)
    _, g = ref.loss_and_grad(params, L, sp, sc, y)
    # finite differences on the head (no rounding points downstream of it)
    n = 3 * L ** 3 * 2
    for i in (16512, 16513, 16470):
        h = 1e-2
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        lp, _ = ref.loss_and_grad(pp, L, sp, sc, y)
        lm, _ = ref.loss_and_grad(pm, L, sp, sc, y)
        assert abs((lp - lm) / (2 * h) / n - g[i]) < 1e-3 * max(1.0, abs(g[i]))


def test_convolution_matches_direct_loop():
    """The reference's periodic convolution is out(r) = sum_k W[co][ci][k] in(r + offset_k),
    offset of k = (kz, ky, kx) = (dz + 1, dy + 1, dx + 1), written out as loops in binary64."""
    L, CI, CO = 5, 3, 2
    rng = np.random.default_rng(0)
    x = rng.normal(size=(1, CI, L, L, L))
    w = rng.normal(size=(CO, CI, 3, 3, 3))
    got = ref._conv(torch.from_numpy(x).float(), torch.from_numpy(w).float()).numpy()[0]
    for (z, y, xx) in [(0, 0, 0), (4, 4, 4), (2, 0, 3), (1, 4, 0)]:
        for co in range(CO):
            acc = 0.0
            for ci in range(CI):
                for kz in range(3):
                    for ky in range(3):
                        for kx in range(3):
                            acc += w[co, ci, kz, ky, kx] * x[0, ci, (z + kz - 1) % L, (y + ky - 1) % L,
                                                              (xx + kx - 1) % L]
            assert abs(got[co, z, y, xx] - acc) < 1e-4 * (1 + abs(acc))


def test_feature_channels_follow_the_documented_order():
    """Channel c < 3 of site r is s_{t-1}(face c, r), channel 3 + c is s_t(face c, r)."""
    L, S = 3, 2
    n = 3 * L ** 3
    sp = inp.random_bits(S, n, 0.3, 5)
    sc = inp.random_bits(S, n, 0.3, 6)
    f = ref.features(L, sp, sc).numpy()
    for s in range(S):
        for c in range(3):
            for site in (0, 7, L ** 3 - 1):
                z, y, x = site // (L * L), (site // L) % L, site % L
                assert f[s, c, z, y, x] == sp[s, c * L ** 3 + site]
                assert f[s, 3 + c, z, y, x] == sc[s, c * L ** 3 + site]
