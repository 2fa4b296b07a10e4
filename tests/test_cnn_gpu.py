"""Warm-start network kernels (BF16 operands, FP32 accumulation) against the float64 CPU oracle,
through the C ABI: forward, backward, loss, optimiser step and patch extraction.

The GPU rounds weights and inputs to BF16 (8 significant bits) and every activation between
layers too; the oracle is given the same BF16 weights and inputs, so what remains is the rounding
of the four hidden activations (relative 2^-9 each) and of the input-gradients in the backward
pass: outputs are compared to 3 % of their scale, gradients per parameter block by relative norm
(3 % for the dense layers, 10 % for the convolutions, whose gradients pass through more BF16
input-gradient roundings) and direction (cosine >= 0.995).  (The oracle makes float64 the default dtype, so every
tensor handed to the kernels here names its dtype.)"""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import cnn_oracle as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1611_03404_gb300 as pkg
    from paper_1611_03404_gb300 import cnn
    return pkg, cnn


def _bf16_bits(t):
    return t.to(torch.bfloat16).view(torch.int16).contiguous()


def _from_bits(b):
    return b.view(torch.bfloat16).to(torch.float64).cpu()


def test_param_count(P):
    pkg, cnn = P
    assert pkg.lib().celeste_cnn_param_count() == C.N_PARAMS


def test_forward_and_backward_match_oracle(P):
    pkg, cnn = P
    dev = torch.device("cuda:0")
    net = cnn.WarmStartCNN(dev, seed=11)
    # biases away from zero so that every ReLU sees both signs
    net.params += 0.05 * torch.randn(net.n, device=dev, dtype=torch.float32,
                                     generator=torch.Generator(device=dev).manual_seed(1))
    net.params_bf16.copy_(_bf16_bits(net.params))
    B = 64
    x = _bf16_bits(torch.randn(B, 32, 32, 5, device=dev, dtype=torch.float32,
                               generator=torch.Generator(device=dev).manual_seed(2)))
    y = net.forward(x)
    pw = _from_bits(net.params_bf16)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in C.SHAPES])
    for k, (name, _) in enumerate(C.SHAPES):      # biases are read in FP32
        if name.startswith("b"):
            pw[offs[k]:offs[k + 1]] = net.params[offs[k]:offs[k + 1]].double().cpu()
    xr = _from_bits(x)
    yr = C.forward(pw, xr)
    scale = float(yr.pow(2).mean().sqrt())
    assert float((y.double().cpu() - yr).abs().max()) <= 3e-2 * scale
    # backward of sum(y * dy) against the oracle's gradient of the same function
    dy = torch.randn(B, 27, device=dev, dtype=torch.float32, generator=torch.Generator(device=dev).manual_seed(3))
    net.grad.zero_()
    net.backward(x, dy)
    p = pw.clone().requires_grad_(True)
    (gr,) = torch.autograd.grad((C.forward(p, xr) * dy.double().cpu()).sum(), p)
    g = net.grad.double().cpu()
    errs = {}
    for k, (name, _) in enumerate(C.SHAPES):
        a, b = g[offs[k]:offs[k + 1]], gr[offs[k]:offs[k + 1]]
        errs[name] = (float((a - b).norm() / b.norm()), float(a @ b / (a.norm() * b.norm())))
    print("CNN_GRAD " + " ".join(f"{n}:{r:.3g}/{c:.5f}" for n, (r, c) in errs.items()))
    # the last layer's gradient sees one rounding, the first layer's every input-gradient pass of the
    # four layers above it (plus ReLU masks that flip where a pre-activation rounds across zero)
    for name, (rel, cos) in errs.items():
        lim = 3e-2 if name in ("w6", "b6", "w5", "b5") else 1e-1
        assert rel <= lim and cos >= 0.995, (name, rel, cos)


def test_mse_and_adamw_match_oracle(P):
    pkg, cnn = P
    dev = torch.device("cuda:0")
    net = cnn.WarmStartCNN(dev, seed=5)
    gen = torch.Generator(device=dev).manual_seed(4)
    f32 = dict(device=dev, dtype=torch.float32, generator=gen)
    y = torch.randn(37, 27, **f32)
    t = torch.randn(37, 27, **f32)
    w = torch.rand(27, **f32) + 0.5
    loss, dy = net.mse(y, t, w)
    yd, td, wd = (a.double().cpu().requires_grad_(a is y) for a in (y, t, w))
    L = C.mse(yd, td, wd)
    (gref,) = torch.autograd.grad(L, yd)
    assert abs(float(loss) - float(L.detach())) <= 1e-6 * float(L.detach())
    assert float((dy.double().cpu() - gref).abs().max()) <= 1e-6 * float(gref.abs().max())
    # two AdamW steps
    p0 = net.params.double().cpu().numpy()
    m = np.zeros_like(p0)
    v = np.zeros_like(p0)
    for step in (1, 2):
        g = torch.randn(net.n, **f32)
        net.grad.copy_(g)
        net.adamw(1e-3, weight_decay=0.01)
        p0, m, v = C.adamw_step(p0, m, v, g.double().cpu().numpy(), 1e-3, 0.9, 0.999, 1e-8, 0.01, step)
    np.testing.assert_allclose(net.params.double().cpu().numpy(), p0, rtol=1e-5, atol=1e-7)
    np.testing.assert_array_equal(net.params_bf16.cpu().numpy(), _bf16_bits(net.params).cpu().numpy())


def test_patch_extraction_matches_oracle(P):
    pkg, cnn = P
    dev = torch.device("cuda:0")
    sc = synth.tiny(seed=3, n_sources=4, n_images=4, H=50, W=56, rotate=True)
    prob = pkg.Problem(sc, device=dev)
    x = _from_bits(prob.extract_patches()).numpy()
    cen = C.patch_centres(sc)
    for s in range(sc.n_sources):
        ref = C.extract_patch(sc, s, cen)
        assert np.all(np.abs(x[s] - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-6), s


@pytest.mark.parametrize("B", [300, 4096])
def test_tcgen05_forward_matches_mma_sync_and_oracle(P, B):
    """The forward pass on the tcgen05 tensor cores (tensor-memory accumulator, 128-row tiles) against
    the warp-level mma.sync engine and the float64 oracle: the same BF16 operands and FP32
    accumulation, so the two engines differ only in summation order (the first layer's BF16
    activations within a few units in the last place, the outputs within 1e-2 of their scale), and
    both stay within the oracle test's 3 % of the output scale.  B = 300 leaves partial last tiles in
    the dense layers and the last convolution."""
    pkg, cnn = P
    dev = torch.device("cuda:0")
    net = cnn.WarmStartCNN(dev, seed=13)
    net.params += 0.05 * torch.randn(net.n, device=dev, dtype=torch.float32,
                                     generator=torch.Generator(device=dev).manual_seed(4))
    net.params_bf16.copy_(_bf16_bits(net.params))
    x = _bf16_bits(torch.randn(B, 32, 32, 5, device=dev, dtype=torch.float32,
                               generator=torch.Generator(device=dev).manual_seed(5)))
    y_ref = net.forward(x, engine=cnn.ENGINE_MMA_SYNC)
    a1_ref = net.buffers(B)["a1"].clone()
    y_tc = net.forward(x, engine=cnn.ENGINE_TCGEN05)
    torch.cuda.synchronize()
    assert pkg.lib().celeste_cnn_status() == 0
    a1_tc = net.buffers(B)["a1"].clone()
    a_ref = a1_ref.view(torch.bfloat16).float()
    a_tc = a1_tc.view(torch.bfloat16).float()
    assert float((a_tc - a_ref).abs().max()) <= 2 ** -6 * float(a_ref.abs().max())
    assert float((a_tc - a_ref).norm() / a_ref.norm()) <= 2e-3
    scale = float(y_ref.double().pow(2).mean().sqrt())
    assert float((y_tc.double() - y_ref.double()).abs().max()) <= 1e-2 * scale
    # against the oracle on a sample of the batch
    pw = _from_bits(net.params_bf16)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in C.SHAPES])
    for k, (name, _) in enumerate(C.SHAPES):
        if name.startswith("b"):
            pw[offs[k]:offs[k + 1]] = net.params[offs[k]:offs[k + 1]].double().cpu()
    idx = torch.arange(0, B, max(1, B // 64))
    yr = C.forward(pw, _from_bits(x[idx.to(dev)]))
    s_or = float(yr.pow(2).mean().sqrt())
    assert float((y_tc[idx.to(dev)].double().cpu() - yr).abs().max()) <= 3e-2 * s_or


def test_backward_layer_by_layer_matches_oracle(P):
    """Each layer's weight and input gradient against the float64 oracle fed the GPU's own BF16
    operands: the layer's input activation (the input patch for the first layer) and the gradient
    w.r.t. its pre-ReLU output as the backward pass left them in the workspace.  What remains is the
    FP32 summation order (weights: 1e-4 of the gradient's norm) and the BF16 rounding of each stored
    input gradient (2^-8 of its scale), so each layer is checked at its own precision rather than
    through the roundings of every layer above it."""
    pkg, cnn = P
    dev = torch.device("cuda:0")
    net = cnn.WarmStartCNN(dev, seed=17)
    net.params += 0.05 * torch.randn(net.n, device=dev, dtype=torch.float32,
                                     generator=torch.Generator(device=dev).manual_seed(6))
    net.params_bf16.copy_(_bf16_bits(net.params))
    B = 96
    x = _bf16_bits(torch.randn(B, 32, 32, 5, device=dev, dtype=torch.float32,
                               generator=torch.Generator(device=dev).manual_seed(7)))
    net.forward(x)
    dy = torch.randn(B, 27, device=dev, dtype=torch.float32, generator=torch.Generator(device=dev).manual_seed(8))
    net.grad.zero_()
    net.backward(x, dy)
    torch.cuda.synchronize()
    buf = {k: _from_bits(v) for k, v in net.buffers(B).items()}
    pw = _from_bits(net.params_bf16)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in C.SHAPES])
    names = [n for n, _ in C.SHAPES]
    for k, (name, _) in enumerate(C.SHAPES):
        if name.startswith("b"):
            pw[offs[k]:offs[k + 1]] = net.params[offs[k]:offs[k + 1]].double().cpu()
    g = net.grad.double().cpu()
    inputs = {1: _from_bits(x), 2: buf["a1"], 3: buf["a2"], 4: buf["a3"], 5: buf["a4"], 6: buf["a5"]}
    out_grads = {k: buf[f"d{k}"] for k in range(1, 6)}
    # the last layer's products take the FP32 output gradient rounded to BF16; its bias gradient sums
    # it unrounded
    out_grads[6] = _from_bits(_bf16_bits(dy))
    report = {}
    for k in range(1, 7):
        p = pw.clone().requires_grad_(True)
        xin = inputs[k].clone().requires_grad_(True)
        z = C.layer_pre(p, k, xin)
        (gp, gx) = torch.autograd.grad((z * out_grads[k].reshape(z.shape)).sum(), (p, xin))
        if k == 6:
            gp = gp.clone()
            gp[offs[names.index("b6")]:offs[names.index("b6") + 1]] = dy.double().cpu().sum(0)
        iw, ib = names.index(f"w{k}"), names.index(f"b{k}")
        for idx in (iw, ib):
            a, b = g[offs[idx]:offs[idx + 1]], gp[offs[idx]:offs[idx + 1]]
            rel = float((a - b).norm() / b.norm())
            report[names[idx]] = rel
            assert rel <= 1e-4, (names[idx], rel)
        if k >= 2:
            # the gradient w.r.t. layer k-1's pre-ReLU value: this input gradient masked by the ReLU
            ref = gx.reshape(out_grads[k - 1].shape) * (inputs[k].reshape(out_grads[k - 1].shape) > 0)
            got = out_grads[k - 1]
            err = float((got - ref).abs().max())
            report[f"d{k - 1}"] = err / float(ref.abs().max())
            assert err <= 2.0 ** -8 * float(ref.abs().max()), (k, err, float(ref.abs().max()))
    print("CNN_LAYER_GRAD " + " ".join(f"{n}:{v:.2e}" for n, v in report.items()))
