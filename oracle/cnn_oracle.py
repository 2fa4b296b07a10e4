"""FP64 CPU oracle for the learned warm start.  TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may import this
module.  It shares no code with the CUDA path.

What it computes: the warm-start network (a small CNN from a source's 5-band 32 x 32 patch to
its 27 initial parameters, which Newton then refines to the same tolerance), its input patch,
the mean-squared-error loss of the standardised targets and one AdamW step, written out in plain
float64 with PyTorch's convolution and linear primitives (library routines used as single steps;
gradients by automatic differentiation).

Network: conv3x3 5->32 stride 1, then 32->64, 64->64, 64->64 stride 2, padding 1, ReLU; the
4 x 4 x 64 map flattened in (h, w, c) order; fully connected 1024->256, ReLU, 256->27.
Parameter vector: W1 [32][3][3][5], b1, W2 [64][3][3][32], b2, W3 [64][3][3][64], b3,
W4 [64][3][3][64], b4, W5 [256][1024], b5, W6 [27][256], b6 (weights indexed [out][kh][kw][in]).
"""
import math

import numpy as np
import torch
import torch.nn.functional as F

SHAPES = [("w1", (32, 3, 3, 5)), ("b1", (32,)), ("w2", (64, 3, 3, 32)), ("b2", (64,)),
          ("w3", (64, 3, 3, 64)), ("b3", (64,)), ("w4", (64, 3, 3, 64)), ("b4", (64,)),
          ("w5", (256, 1024)), ("b5", (256,)), ("w6", (27, 256)), ("b6", (27,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p):
    """Named views of the flat parameter vector."""
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def forward(p, x):
    """p: float64 [N_PARAMS]; x: float64 [B, 32, 32, 5] (NHWC) -> [B, 27]."""
    w = unpack(p)
    h = x.permute(0, 3, 1, 2)                                     # NCHW for the library routine
    for k, stride in ((1, 1), (2, 2), (3, 2), (4, 2)):
        wk = w[f"w{k}"].permute(0, 3, 1, 2)                       # [out][in][kh][kw]
        h = F.relu(F.conv2d(h, wk, w[f"b{k}"], stride=stride, padding=1))
    h = h.permute(0, 2, 3, 1).reshape(h.shape[0], -1)             # flatten in (h, w, c) order
    h = F.relu(F.linear(h, w["w5"], w["b5"]))
    return F.linear(h, w["w6"], w["b6"])


def layer_pre(p, k, x):
    """Layer k's pre-activation (before ReLU) from its input x: k = 1..4 the convolutions (x NHWC
    [B, H, W, C] -> NHWC), k = 5, 6 the dense layers (x [B, 1024] or [B, 256]; for k = 5 a 4 x 4 x 64
    map is flattened in (h, w, c) order).  The same arithmetic as `forward`, one layer at a time."""
    w = unpack(p)
    if k <= 4:
        stride = 1 if k == 1 else 2
        h = F.conv2d(x.permute(0, 3, 1, 2), w[f"w{k}"].permute(0, 3, 1, 2), w[f"b{k}"], stride=stride, padding=1)
        return h.permute(0, 2, 3, 1)
    return F.linear(x.reshape(x.shape[0], -1), w[f"w{k}"], w[f"b{k}"])


def mse(y, t, weight=None):
    """Mean over [B, 27] of weight_j (y - t)^2."""
    d = (y - t) ** 2
    if weight is not None:
        d = d * weight
    return d.mean()


def loss_and_grad(p, x, t, weight=None):
    p = p.clone().requires_grad_(True)
    L = mse(forward(p, x), t, weight)
    (g,) = torch.autograd.grad(L, p)
    return float(L), g


def adamw_step(p, m, v, g, lr, b1, b2, eps, wd, step):
    """Decoupled weight decay, bias-corrected moments."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    p = p * (1 - lr * wd) - lr * mh / (np.sqrt(vh) + eps)
    return p, m, v


def extract_patch(scene, s, radius_centres):
    """Network input of source s: for each band, the first image (in image order) holding the
    source's patch centre; a 32 x 32 window with the centre at (16, 16); asinh((x - sky)/sqrt(sky));
    zero outside the image or for a missing band.  radius_centres[s] = list of (image, cx, cy)."""
    out = np.zeros((32, 32, 5))
    seen = set()
    for (n, cx, cy) in radius_centres[s]:
        im = scene.images[n]
        if im.band in seen:
            continue
        seen.add(im.band)
        for i in range(32):
            r = cy - 16 + i
            if r < 0 or r >= im.H:
                continue
            for j in range(32):
                c = cx - 16 + j
                if 0 <= c < im.W:
                    out[i, j, im.band] = math.asinh((float(im.pixels[r, c]) - im.sky) / math.sqrt(im.sky))
    return out


def patch_centres(scene):
    """Per source: (image, cx, cy) of every image whose pixel grid holds round(A u0 + o)."""
    out = []
    for s in range(scene.n_sources):
        lst = []
        for n, im in enumerate(scene.images):
            p = im.wcs[:4].reshape(2, 2) @ scene.u0[s] + im.wcs[4:]
            cx, cy = math.floor(p[0] + 0.5), math.floor(p[1] + 0.5)
            if 0 <= cx <= im.W - 1 and 0 <= cy <= im.H - 1:
                lst.append((n, cx, cy))
        out.append(lst)
    return out
