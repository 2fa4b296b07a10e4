"""Pins of the warm-start network's CPU oracle: the convolution convention against a direct
loop over the definition, the backward pass against central finite differences of the forward,
the AdamW step against its first-step closed form, the patch extraction against the image."""
import math

import numpy as np
import torch

import synth
from oracle import cnn_oracle as C


def _params(seed, scale=0.2):
    g = torch.Generator().manual_seed(seed)
    return torch.randn(C.N_PARAMS, generator=g, dtype=torch.float64) * scale


def test_param_count():
    assert C.N_PARAMS == 32 * 45 + 32 + 64 * 288 + 64 + 2 * (64 * 576 + 64) + 256 * 1024 + 256 + 27 * 256 + 27


def test_first_conv_matches_direct_loop():
    """out[b, oh, ow, co] = relu(b[co] + sum_{kh,kw,ci} x[b, oh + kh - 1, ow + kw - 1, ci] W[co, kh, kw, ci]),
    checked through the first layer (stride 1) and, with a stride-2 layer on top, at the border."""
    p = _params(1)
    w = C.unpack(p)
    x = torch.randn(1, 32, 32, 5, generator=torch.Generator().manual_seed(2), dtype=torch.float64)
    h1 = torch.relu(torch.nn.functional.conv2d(x.permute(0, 3, 1, 2), w["w1"].permute(0, 3, 1, 2), w["b1"],
                                               padding=1)).permute(0, 2, 3, 1)
    for (oh, ow, co) in [(0, 0, 3), (5, 31, 0), (17, 9, 31), (31, 31, 12)]:
        v = float(w["b1"][co])
        for kh in range(3):
            for kw in range(3):
                ih, iw = oh + kh - 1, ow + kw - 1
                if 0 <= ih < 32 and 0 <= iw < 32:
                    v += float((x[0, ih, iw, :] * w["w1"][co, kh, kw, :]).sum())
        assert abs(max(v, 0.0) - float(h1[0, oh, ow, co])) <= 1e-12 * (1 + abs(v))
    # stride 2: output (oh, ow) reads input rows 2 oh - 1 .. 2 oh + 1
    h2 = torch.relu(torch.nn.functional.conv2d(h1.permute(0, 3, 1, 2), w["w2"].permute(0, 3, 1, 2), w["b2"],
                                               stride=2, padding=1)).permute(0, 2, 3, 1)
    for (oh, ow, co) in [(0, 0, 1), (15, 7, 63)]:
        v = float(w["b2"][co])
        for kh in range(3):
            for kw in range(3):
                ih, iw = 2 * oh + kh - 1, 2 * ow + kw - 1
                if 0 <= ih < 32 and 0 <= iw < 32:
                    v += float((h1[0, ih, iw, :] * w["w2"][co, kh, kw, :]).sum())
        assert abs(max(v, 0.0) - float(h2[0, oh, ow, co])) <= 1e-12 * (1 + abs(v))


def test_flatten_order_and_head():
    """The 4 x 4 x 64 map enters the first dense layer in (h, w, c) order: moving one weight of
    W5 column (h * 4 + w) * 64 + c changes the output exactly through that activation."""
    p = _params(3)
    x = torch.randn(2, 32, 32, 5, generator=torch.Generator().manual_seed(4), dtype=torch.float64)
    y0 = C.forward(p, x)
    assert y0.shape == (2, 27)
    w = C.unpack(p)
    # activation a4 via the layers alone
    h = x.permute(0, 3, 1, 2)
    for k, s in ((1, 1), (2, 2), (3, 2), (4, 2)):
        h = torch.relu(torch.nn.functional.conv2d(h, w[f"w{k}"].permute(0, 3, 1, 2), w[f"b{k}"], stride=s, padding=1))
    a4 = h.permute(0, 2, 3, 1)                                    # [B, 4, 4, 64]
    hh, ww, cc = 2, 1, 37
    col = (hh * 4 + ww) * 64 + cc
    assert float(a4[0, hh, ww, cc]) > 0.0   # the probed activation is live for this seed
    off = 32 * 45 + 32 + 64 * 288 + 64 + 2 * (64 * 576 + 64)
    q = p.clone()
    q[off + 5 * 1024 + col] += 1e-3                               # W5[5][col]
    a5 = torch.relu(torch.nn.functional.linear(a4.reshape(2, -1), w["w5"], w["b5"]))
    assert float(a5[0, 5]) > 0.0
    dy = C.forward(q, x)[0] - y0[0]
    expect = 1e-3 * float(a4[0, hh, ww, cc]) * w["w6"][:, 5]
    assert torch.allclose(dy, expect, rtol=1e-6, atol=1e-12)


def test_backward_matches_finite_differences():
    p = _params(5, 0.15)
    x = torch.randn(3, 32, 32, 5, generator=torch.Generator().manual_seed(6), dtype=torch.float64)
    t = torch.randn(3, 27, generator=torch.Generator().manual_seed(7), dtype=torch.float64)
    wt = torch.rand(27, generator=torch.Generator().manual_seed(8), dtype=torch.float64) + 0.5
    L, g = C.loss_and_grad(p, x, t, wt)
    rng = np.random.default_rng(9)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in C.SHAPES])
    idx = [int(rng.integers(offs[k], offs[k + 1])) for k in range(len(C.SHAPES))]
    for i in idx:
        h = 1e-6
        e = torch.zeros_like(p)
        e[i] = h
        fd = (float(C.mse(C.forward(p + e, x), t, wt)) - float(C.mse(C.forward(p - e, x), t, wt))) / (2 * h)
        assert abs(fd - float(g[i])) <= 1e-6 * max(1e-3, abs(fd)), (i, fd, float(g[i]))


def test_adamw_first_step_closed_form():
    """After one step from zero moments the bias-corrected update is lr * g / (|g| + eps) per entry."""
    p = np.array([0.5, -1.0, 2.0])
    g = np.array([0.1, -3.0, 1e-9])
    lr, wd = 1e-2, 0.1
    q, m, v = C.adamw_step(p, np.zeros(3), np.zeros(3), g, lr, 0.9, 0.999, 1e-8, wd, 1)
    np.testing.assert_allclose(q, p * (1 - lr * wd) - lr * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_patch_extraction_reads_the_image():
    sc = synth.tiny(seed=3, n_sources=2, n_images=3, H=40, W=44, rotate=False)
    cen = C.patch_centres(sc)
    for s in range(sc.n_sources):
        x = C.extract_patch(sc, s, cen)
        n, cx, cy = cen[s][0]
        im = sc.images[n]
        assert x[16, 16, im.band] == math.asinh((float(im.pixels[cy, cx]) - im.sky) / math.sqrt(im.sky))
        bands = {sc.images[m].band for (m, _, _) in cen[s]}
        for b in set(range(5)) - bands:
            assert not x[:, :, b].any()


def test_layer_pre_composes_to_forward():
    """layer_pre, one layer at a time, composed with ReLU between layers, is the network's forward
    (which the tests above pin against a direct loop over the convolution's definition and finite
    differences), and each convolution layer's output has the stride's spatial size."""
    rng = np.random.default_rng(12)
    p = torch.as_tensor(rng.standard_normal(C.N_PARAMS) * 0.05)
    x = torch.as_tensor(rng.standard_normal((3, 32, 32, 5)))
    h = x
    for k, side in zip(range(1, 5), (32, 16, 8, 4)):
        h = torch.relu(C.layer_pre(p, k, h))
        assert tuple(h.shape) == (3, side, side, 32 if k == 1 else 64)
    h = torch.relu(C.layer_pre(p, 5, h))
    y = C.layer_pre(p, 6, h)
    np.testing.assert_allclose(y.numpy(), C.forward(p, x).numpy(), rtol=1e-12, atol=1e-12)
