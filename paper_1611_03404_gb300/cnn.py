"""Learned warm start (argument marshalling around the library's CNN kernels).

WarmStartCNN holds the network's FP32 master parameters, their BF16 copy and the AdamW moments as
device tensors; forward, backward, loss and optimiser steps are the library's kernels
(include/celeste.h).  Training targets are the converged parameters of earlier solves, with the
position given as the offset from the catalog position and every column standardised; the
network's last layer maps back to parameter space in its epilogue.

warm_start() builds a Newton starting point from the catalog and the prediction: the network
supplies the quantities the catalog does not carry (type probability, the variational variances
of flux and colours), the catalog keeps position, shape, flux and colour means unless asked
otherwise.
"""
import ctypes

import numpy as np
import torch

from .celeste import NPARAM, _check, _ptr, _stream, lib

PATCH = 32
BANDS = 5
ENGINE_MMA_SYNC, ENGINE_TCGEN05 = 0, 1
# parameters taken from the network by default (indices in the 27-vector): the type logit (6)
# and the log variances of the log fluxes (8, 10) and of the colours (15-18, 23-26), which the
# catalog does not carry; position, shape, flux and colour means stay the catalog's
NET_PARAMS = [6, 8, 10] + list(range(15, 19)) + list(range(23, 27))


def _aligned(nbytes, device):
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return buf, ctypes.c_void_p(buf.data_ptr() + off), nbytes


class WarmStartCNN:
    def __init__(self, device="cuda", seed=0):
        L = lib()
        self.device = torch.device(device)
        self.n = int(L.celeste_cnn_param_count())
        self.params = torch.empty(self.n, dtype=torch.float32, device=self.device)
        self.params_bf16 = torch.empty(self.n, dtype=torch.int16, device=self.device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.step = 0
        self.mu = torch.zeros(NPARAM, dtype=torch.float32, device=self.device)
        self.sd = torch.ones(NPARAM, dtype=torch.float32, device=self.device)
        self._ws = {}
        _check(L.celeste_cnn_init(_ptr(self.params), _ptr(self.params_bf16), ctypes.c_uint64(seed), _stream(None)))

    def workspace(self, batch):
        if batch not in self._ws:
            self._ws[batch] = _aligned(int(lib().celeste_cnn_workspace_bytes(batch)), self.device)
        return self._ws[batch]

    def forward(self, x, standardised=True, engine=None):
        """x: int16 [B, 32, 32, 5] (BF16 bits) -> [B, 27] float32 (standardised, or parameter space).
        engine: None (the library's default), ENGINE_MMA_SYNC or ENGINE_TCGEN05."""
        assert x.dtype == torch.int16 and x.is_contiguous() and tuple(x.shape[1:]) == (PATCH, PATCH, BANDS)
        B = x.shape[0]
        y = torch.empty(B, NPARAM, dtype=torch.float32, device=self.device)
        _, ws, nb = self.workspace(B)
        sc, sh = (None, None) if standardised else (self.sd, self.mu)
        if engine is None:
            _check(lib().celeste_cnn_forward(_ptr(self.params), _ptr(self.params_bf16), _ptr(x), B, _ptr(sc),
                                             _ptr(sh), _ptr(y), ws, ctypes.c_size_t(nb), _stream(None)))
        else:
            _check(lib().celeste_cnn_forward_ex(_ptr(self.params), _ptr(self.params_bf16), _ptr(x), B, _ptr(sc),
                                                _ptr(sh), _ptr(y), ws, ctypes.c_size_t(nb), ctypes.c_int(engine),
                                                _stream(None)))
        return y

    def buffers(self, batch):
        """The workspace's BF16 buffers (int16 bit patterns) at this batch size: a1..a5, the five hidden
        layers' activations after ReLU kept by the last forward call, and d1..d5, the gradients w.r.t.
        their pre-ReLU values left by the last backward call (the library's workspace layout: a_k then
        d_k for k = 1..5, each 256-byte aligned)."""
        buf, ws, _ = self.workspace(batch)
        off = ws.value - buf.data_ptr()
        shapes = [(32, 32, 32), (16, 16, 64), (8, 8, 64), (4, 4, 64), (256,)]
        out = {}
        for k, shp in enumerate(shapes, 1):
            n = batch * int(np.prod(shp))
            for name in ("a", "d"):
                out[f"{name}{k}"] = buf[off:off + 2 * n].view(torch.int16).view(batch, *shp)
                off += (2 * n + 255) // 256 * 256
        return out

    def backward(self, x, dy):
        assert x.dtype == torch.int16 and dy.dtype == torch.float32 and dy.is_contiguous()
        B = x.shape[0]
        _, ws, nb = self.workspace(B)
        _check(lib().celeste_cnn_backward(_ptr(self.params), _ptr(self.params_bf16), _ptr(x), _ptr(dy), B,
                                          _ptr(self.grad), ws, ctypes.c_size_t(nb), _stream(None)))

    def mse(self, y, target, weight=None):
        assert y.dtype == target.dtype == torch.float32 and y.is_contiguous() and target.is_contiguous()
        assert weight is None or (weight.dtype == torch.float32 and weight.numel() == NPARAM)
        B = y.shape[0]
        dy = torch.empty_like(y)
        loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        _check(lib().celeste_cnn_mse(_ptr(y), _ptr(target), _ptr(weight), B, _ptr(dy), _ptr(loss), _stream(None)))
        return loss, dy

    def adamw(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=1e-4):
        assert self.grad.dtype == torch.float32
        self.step += 1
        _check(lib().celeste_cnn_adamw(_ptr(self.params), _ptr(self.params_bf16), _ptr(self.m), _ptr(self.v),
                                       _ptr(self.grad), ctypes.c_float(lr), ctypes.c_float(beta1),
                                       ctypes.c_float(beta2), ctypes.c_float(eps), ctypes.c_float(weight_decay),
                                       self.step, _stream(None)))

    def set_standardisation(self, targets):
        """Column means and deviations of the training targets (parameter space, offsets for u)."""
        self.mu = targets.mean(0).float().contiguous()
        self.sd = targets.std(0).clamp_min(1e-3).float().contiguous()

    def train(self, x, targets, epochs=10, batch=512, lr=2e-3, weight_decay=1e-4, seed=0, weight=None):
        """x: int16 [N, 32, 32, 5]; targets: float [N, 27] in parameter space (u as offsets).
        Returns the mean loss of every epoch."""
        self.set_standardisation(targets)
        # standardised targets clipped at 5 deviations: weakly identified parameters (a star's
        # galaxy shape, say) can sit far out and would otherwise dominate the loss
        t = ((targets.float() - self.mu) / self.sd).clamp(-5.0, 5.0).contiguous()
        N = x.shape[0]
        gen = torch.Generator(device=self.device)
        gen.manual_seed(seed)
        history = []
        steps_per_epoch = max(1, N // batch)
        total = epochs * steps_per_epoch
        for ep in range(epochs):
            perm = torch.randperm(N, device=self.device, generator=gen)
            acc = torch.zeros(1, dtype=torch.float64, device=self.device)
            for i in range(steps_per_epoch):
                idx = perm[i * batch:(i + 1) * batch]
                xb, tb = x[idx].contiguous(), t[idx].contiguous()
                y = self.forward(xb)
                loss, dy = self.mse(y, tb, weight)
                self.grad.zero_()
                self.backward(xb, dy)
                k = ep * steps_per_epoch + i
                cur = lr * 0.5 * (1.0 + np.cos(np.pi * k / total))   # cosine schedule
                self.adamw(cur, weight_decay=weight_decay)
                acc += loss
            history.append(float(acc) / steps_per_epoch)
        return history

    def predict(self, x, batch=4096):
        """Parameter-space predictions (u as offsets) for every row of x."""
        out = []
        for i in range(0, x.shape[0], batch):
            out.append(self.forward(x[i:i + batch].contiguous(), standardised=False))
        return torch.cat(out, 0)


def training_targets(theta_star, u0):
    """Converged parameters with the position replaced by its offset from the catalog position."""
    t = theta_star.clone()
    t[:, 0:2] -= u0
    return t


def warm_start(theta_catalog, prediction, params=NET_PARAMS):
    """Newton starting point: the catalog with the listed parameters taken from the prediction
    (a prediction of u is an offset from the catalog position)."""
    th = theta_catalog.clone()
    for j in params:
        th[:, j] = prediction[:, j] + (theta_catalog[:, j] if j < 2 else 0.0)
    return th.contiguous()
