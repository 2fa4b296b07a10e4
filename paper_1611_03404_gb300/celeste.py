"""Thin ctypes binding of the C ABI in include/celeste.h (argument marshalling only).

Every step of the computation runs in the CUDA library; this module converts Python /
torch arguments into the plain pointers and sizes the C functions take, and raises on
error codes.  There is no fallback: if the library is missing, importing fails loudly.
"""
import ctypes
import os

import numpy as np
import torch

from . import build as _build

NPARAM = 27
WANT_ELBO, WANT_GRAD, WANT_HESS = 1, 2, 4
STATUS_CONVERGED, STATUS_MAX_ITER, STATUS_NONFINITE, STATUS_RADIUS_COLLAPSE = 0, 1, 2, 3
HESS_FP32, HESS_TF32, HESS_BF16X3, HESS_BF16X6, HESS_TF32X3 = 0, 1, 2, 3, 4
NBR_FULL, NBR_WINDOW = 0, 1


class CelesteError(RuntimeError):
    pass


class ImageDesc(ctypes.Structure):
    _fields_ = [("height", ctypes.c_int32), ("width", ctypes.c_int32), ("band", ctypes.c_int32),
                ("pixels", ctypes.c_void_p), ("sky", ctypes.c_double), ("iota", ctypes.c_double),
                ("wcs", ctypes.c_double * 6), ("psf", ctypes.c_double * 108)]


class ProblemDesc(ctypes.Structure):
    _fields_ = [("n_images", ctypes.c_int32), ("images", ctypes.POINTER(ImageDesc)),
                ("n_sources", ctypes.c_int32), ("u0", ctypes.POINTER(ctypes.c_double)),
                ("radius", ctypes.POINTER(ctypes.c_int32)), ("priors", ctypes.c_double * 5),
                ("exp_nu", ctypes.c_double * 6), ("exp_tau", ctypes.c_double * 6),
                ("dev_nu", ctypes.c_double * 8), ("dev_tau", ctypes.c_double * 8),
                ("tile_pixels", ctypes.c_int32), ("hessian_mode", ctypes.c_int32)]


class NewtonOpts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("ftol", ctypes.c_double), ("gtol", ctypes.c_double),
                ("delta0", ctypes.c_double), ("delta_max", ctypes.c_double), ("eta", ctypes.c_double),
                ("delta_min", ctypes.c_double), ("graph_iters", ctypes.c_int32), ("cta_sources", ctypes.c_int32)]


class ProfileStats(ctypes.Structure):
    _fields_ = [("full_ms", ctypes.c_double), ("value_ms", ctypes.c_double), ("full_launches", ctypes.c_int64),
                ("value_launches", ctypes.c_int64), ("full_pixels", ctypes.c_int64), ("value_pixels", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("newton_iterations", ctypes.c_int64),
                ("tr_ms", ctypes.c_double), ("tr_launches", ctypes.c_int64)]


EXPORTED = ["celeste_problem_create", "celeste_problem_workspace_bytes", "celeste_problem_counts",
            "celeste_problem_bind", "celeste_render_background", "celeste_elbo_batch", "celeste_newton_batch",
            "celeste_problem_destroy", "celeste_strerror", "celeste_last_error_detail", "celeste_profile_start",
            "celeste_profile_stop", "celeste_tr_solve_batch", "celeste_tr_solve_batch_ex", "celeste_tr_reciprocal", "celeste_elbo_batch_noalloc", "celeste_cnn_param_count",
            "celeste_cnn_workspace_bytes", "celeste_cnn_init", "celeste_cnn_forward", "celeste_cnn_backward",
            "celeste_cnn_mse", "celeste_cnn_adamw", "celeste_extract_patches", "celeste_covariance_batch",
            "celeste_render_background_mode", "celeste_joint_pairs", "celeste_joint_cross_hessian",
            "celeste_joint_newton", "celeste_joint_value", "celeste_problem_check", "celeste_problem_set_wait_budget",
            "celeste_measure_peak", "celeste_joint_workspace_bytes", "celeste_joint_bind", "celeste_cnn_forward_ex",
            "celeste_cnn_status", "celeste_problem_refresh_pixels"]


def load_library(path=None):
    path = path or _build.LIB
    if not os.path.exists(path):
        raise CelesteError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp, i32, u32, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p
    sig = {
        "celeste_problem_create": (ctypes.c_int, [ctypes.POINTER(ProblemDesc), ctypes.POINTER(vp)]),
        "celeste_problem_workspace_bytes": (ctypes.c_size_t, [vp]),
        "celeste_problem_counts": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int64)]),
        "celeste_problem_bind": (ctypes.c_int, [vp, vp, ctypes.c_size_t, vp]),
        "celeste_render_background": (ctypes.c_int, [vp, dp, vp]),
        "celeste_elbo_batch": (ctypes.c_int, [vp, dp, u32, dp, dp, dp, vp]),
        "celeste_newton_batch": (ctypes.c_int, [vp, dp, ctypes.POINTER(NewtonOpts), dp, dp, dp, dp, vp]),
        "celeste_problem_destroy": (None, [vp]),
        "celeste_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "celeste_last_error_detail": (ctypes.c_char_p, []),
        "celeste_profile_start": (ctypes.c_int, [vp]),
        "celeste_profile_stop": (ctypes.c_int, [vp, ctypes.POINTER(ProfileStats)]),
        "celeste_tr_solve_batch": (ctypes.c_int, [dp, dp, dp, ctypes.c_int, dp, dp, dp, vp]),
        "celeste_tr_reciprocal": (ctypes.c_int, [dp, dp, ctypes.c_int, vp]),
        "celeste_tr_solve_batch_ex": (ctypes.c_int, [dp, dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, vp]),
        "celeste_elbo_batch_noalloc": (ctypes.c_int, [vp, dp, dp, dp, dp, vp]),
        "celeste_cnn_param_count": (ctypes.c_int64, []),
        "celeste_cnn_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int]),
        "celeste_cnn_init": (ctypes.c_int, [dp, dp, ctypes.c_uint64, vp]),
        "celeste_cnn_forward": (ctypes.c_int, [dp, dp, dp, ctypes.c_int, dp, dp, dp, dp, ctypes.c_size_t, vp]),
        "celeste_cnn_backward": (ctypes.c_int, [dp, dp, dp, dp, ctypes.c_int, dp, dp, ctypes.c_size_t, vp]),
        "celeste_cnn_mse": (ctypes.c_int, [dp, dp, dp, ctypes.c_int, dp, dp, vp]),
        "celeste_cnn_adamw": (ctypes.c_int, [dp, dp, dp, dp, dp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                             ctypes.c_float, ctypes.c_float, ctypes.c_int, vp]),
        "celeste_extract_patches": (ctypes.c_int, [vp, dp, vp]),
        "celeste_covariance_batch": (ctypes.c_int, [vp, dp, dp, dp, vp]),
        "celeste_render_background_mode": (ctypes.c_int, [vp, dp, ctypes.c_int, vp]),
        "celeste_joint_pairs": (ctypes.c_int, [vp, dp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
        "celeste_joint_cross_hessian": (ctypes.c_int, [vp, dp, dp, vp]),
        "celeste_joint_value": (ctypes.c_int, [vp, dp, ctypes.POINTER(ctypes.c_double), vp]),
        "celeste_problem_check": (ctypes.c_int, [vp, vp]),
        "celeste_problem_set_wait_budget": (ctypes.c_int, [vp, ctypes.c_longlong]),
        "celeste_measure_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                                ctypes.POINTER(ctypes.c_double), vp]),
        "celeste_joint_workspace_bytes": (ctypes.c_size_t, [vp]),
        "celeste_cnn_forward_ex": (ctypes.c_int, [dp, dp, dp, ctypes.c_int, dp, dp, dp, dp, ctypes.c_size_t,
                                                  ctypes.c_int, vp]),
        "celeste_cnn_status": (ctypes.c_int, []),
        "celeste_problem_refresh_pixels": (ctypes.c_int, [vp, vp]),
        "celeste_joint_bind": (ctypes.c_int, [vp, vp, ctypes.c_size_t, vp]),
        "celeste_joint_newton": (ctypes.c_int, [vp, dp, ctypes.POINTER(NewtonOpts), ctypes.c_int32,
                                                ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32), vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


def _check(rc):
    if rc != 0:
        L = lib()
        raise CelesteError(f"{L.celeste_strerror(rc).decode()}: {L.celeste_last_error_detail().decode()}")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Problem:
    """A bound problem: images resident on the device, layout and workspace owned here.

    scene: an object with .images (each .pixels [H,W] float32, .band, .sky, .iota, .wcs[6],
    .psf[3,6,6]), .u0 [S,2], .radius [S], .priors [5] and the exp/deV mixture tables.
    device_pixels: optional list of CUDA float32 tensors already holding the images."""

    def __init__(self, scene, device="cuda", tile_pixels=128, device_pixels=None, stream=None, hessian_mode=0):
        L = lib()
        self.device = torch.device(device)
        if device_pixels is None:
            device_pixels = [torch.as_tensor(np.ascontiguousarray(im.pixels, np.float32)).to(self.device)
                             for im in scene.images]
        self.pixels = [p.contiguous() for p in device_pixels]
        n = len(scene.images)
        self._imgs = (ImageDesc * n)()
        for k, im in enumerate(scene.images):
            d = self._imgs[k]
            d.height, d.width = self.pixels[k].shape
            d.band = int(im.band)
            d.pixels = self.pixels[k].data_ptr()
            d.sky, d.iota = float(im.sky), float(im.iota)
            d.wcs[:] = [float(v) for v in im.wcs]
            d.psf[:] = [float(v) for v in np.asarray(im.psf, np.float64).reshape(-1)]
        self._u0 = np.ascontiguousarray(scene.u0, np.float64)
        self._rad = np.ascontiguousarray(scene.radius, np.int32)
        desc = ProblemDesc()
        desc.n_images = n
        desc.images = self._imgs
        desc.n_sources = self._u0.shape[0]
        desc.u0 = self._u0.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        desc.radius = self._rad.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        desc.priors[:] = [float(v) for v in scene.priors]
        desc.exp_nu[:] = [float(v) for v in scene.exp_nu]
        desc.exp_tau[:] = [float(v) for v in scene.exp_tau]
        desc.dev_nu[:] = [float(v) for v in scene.dev_nu]
        desc.dev_tau[:] = [float(v) for v in scene.dev_tau]
        desc.tile_pixels = int(tile_pixels)
        desc.hessian_mode = int(hessian_mode)
        h = ctypes.c_void_p()
        _check(L.celeste_problem_create(ctypes.byref(desc), ctypes.byref(h)))
        self.handle = h
        self.S = desc.n_sources
        nbytes = L.celeste_problem_workspace_bytes(h)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        off = (-self.workspace.data_ptr()) % 256
        self._ws_ptr = ctypes.c_void_p(self.workspace.data_ptr() + off)
        self._ws_bytes = nbytes
        _check(L.celeste_problem_bind(h, self._ws_ptr, ctypes.c_size_t(nbytes), _stream(stream)))

    def counts(self):
        c = (ctypes.c_int64 * 5)()
        _check(lib().celeste_problem_counts(self.handle, c))
        return dict(sources=c[0], patches=c[1], tiles=c[2], pixels=c[3], neighbours=c[4])

    def render_background(self, nbr_theta, mode=NBR_FULL, stream=None):
        """Neighbour background at nbr_theta; mode NBR_WINDOW counts each neighbour on its own window
        only (the joint objective's per-source blocks)."""
        assert nbr_theta.dtype == torch.float64 and nbr_theta.is_contiguous() and nbr_theta.shape == (self.S, NPARAM)
        _check(lib().celeste_render_background_mode(self.handle, _ptr(nbr_theta), ctypes.c_int(mode), _stream(stream)))

    def joint_pairs(self):
        """[n_pairs, 2] int32 (host numpy): source pairs s < t whose windows overlap."""
        return _joint_pairs(self.handle)

    def _joint_workspace(self, stream=None):
        """Binds the joint calls' device workspace (torch memory) on first use."""
        if getattr(self, "_joint_ws", None) is None:
            L = lib()
            nbytes = L.celeste_joint_workspace_bytes(self.handle)
            buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            off = (-buf.data_ptr()) % 256
            _check(L.celeste_joint_bind(self.handle, ctypes.c_void_p(buf.data_ptr() + off), ctypes.c_size_t(nbytes),
                                        _stream(stream)))
            self._joint_ws = buf

    def joint_newton(self, theta, max_iter=50, ftol=1e-8, gtol=1e-10, delta_max=1e4, eta=0.1, delta_min=1e-12,
                     max_cg=100, stream=None):
        """Trust-region Newton on the joint objective over all sources (theta updated in place).
        Returns dict(iters, status, J, cg_iters)."""
        assert theta.dtype == torch.float64 and theta.is_contiguous() and theta.shape == (self.S, NPARAM)
        self._joint_workspace(stream)
        o = NewtonOpts(max_iter=max_iter, ftol=ftol, gtol=gtol, delta0=1.0, delta_max=delta_max, eta=eta,
                       delta_min=delta_min, graph_iters=1)
        it, st, cg = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
        J = ctypes.c_double(0.0)
        _check(lib().celeste_joint_newton(self.handle, _ptr(theta), ctypes.byref(o), ctypes.c_int32(max_cg),
                                          ctypes.byref(it), ctypes.byref(st), ctypes.byref(J), ctypes.byref(cg),
                                          _stream(stream)))
        return {"iters": it.value, "status": st.value, "J": J.value, "cg_iters": cg.value}

    def joint_value(self, theta, stream=None):
        """The joint objective J at theta (every covered pixel counted once)."""
        assert theta.dtype == torch.float64 and theta.is_contiguous() and theta.shape == (self.S, NPARAM)
        self._joint_workspace(stream)
        J = ctypes.c_double(0.0)
        _check(lib().celeste_joint_value(self.handle, _ptr(theta), ctypes.byref(J), _stream(stream)))
        return J.value

    def cross_hessian(self, theta, stream=None):
        """Cross-source Hessian blocks of the joint objective, [n_pairs, 27, 27] float64 on theta's
        device, in the order of joint_pairs(); the background must be rendered with NBR_WINDOW at theta."""
        assert theta.dtype == torch.float64 and theta.is_contiguous() and theta.shape == (self.S, NPARAM)
        self._joint_workspace(stream)
        n = len(self.joint_pairs())
        out = torch.empty(max(n, 1), NPARAM, NPARAM, dtype=torch.float64, device=theta.device)
        _check(lib().celeste_joint_cross_hessian(self.handle, _ptr(theta), _ptr(out), _stream(stream)))
        return out[:n]

    def elbo_batch(self, theta, want=WANT_ELBO | WANT_GRAD | WANT_HESS, stream=None, check=True):
        """(elbo, grad, hess) per source; with check (default) the stream is synchronised and a device-side
        error (a bulk-copy wait that ran out) raises."""
        assert theta.dtype == torch.float64 and theta.is_contiguous() and theta.shape == (self.S, NPARAM)
        dev = theta.device
        elbo = torch.empty(self.S, dtype=torch.float64, device=dev) if want & WANT_ELBO else None
        grad = torch.empty(self.S, NPARAM, dtype=torch.float64, device=dev) if want & WANT_GRAD else None
        hess = torch.empty(self.S, NPARAM, NPARAM, dtype=torch.float64, device=dev) if want & WANT_HESS else None
        _check(lib().celeste_elbo_batch(self.handle, _ptr(theta), ctypes.c_uint32(want), _ptr(elbo), _ptr(grad),
                                        _ptr(hess), _stream(stream)))
        if check:
            self.check(stream)
        return elbo, grad, hess

    def check(self, stream=None):
        """Waits for the stream; raises CelesteError if the device recorded a timeout or bad pixel counts."""
        _check(lib().celeste_problem_check(self.handle, _stream(stream)))

    def set_wait_budget(self, cycles):
        """Budget (SM cycles) of the pixel kernels' first wait on a tile's bulk copies; 0 restores the default,
        a negative value makes every such wait give up at once (the timeout path, for tests)."""
        _check(lib().celeste_problem_set_wait_budget(self.handle, ctypes.c_longlong(int(cycles))))

    def newton_batch(self, theta, delta=None, max_iter=50, ftol=1e-8, gtol=1e-10, delta0=1.0, delta_max=1e4,
                     eta=0.1, delta_min=1e-12, graph_iters=4, cta_sources=0, stream=None):
        """Runs trust-region Newton in place on `theta`; returns (delta, iters, status, elbo).  cta_sources:
        iterations starting with at most this many active sources solve each subproblem on four warps
        (0: twice the SM count; negative: never)."""
        assert theta.dtype == torch.float64 and theta.is_contiguous() and theta.shape == (self.S, NPARAM)
        dev = theta.device
        if delta is None:
            delta = torch.zeros(self.S, dtype=torch.float64, device=dev)
        iters = torch.zeros(self.S, dtype=torch.int32, device=dev)
        status = torch.zeros(self.S, dtype=torch.int32, device=dev)
        elbo = torch.empty(self.S, dtype=torch.float64, device=dev)
        opts = NewtonOpts(max_iter, ftol, gtol, delta0, delta_max, eta, delta_min, graph_iters, cta_sources)
        _check(lib().celeste_newton_batch(self.handle, _ptr(theta), ctypes.byref(opts), _ptr(delta), _ptr(iters),
                                          _ptr(status), _ptr(elbo), _stream(stream)))
        return delta, iters, status, elbo

    def covariance(self, theta, stream=None):
        """Linear-response covariance (-H)^-1 per source at theta: ([S, 27, 27] float64, ok [S])."""
        assert theta.dtype == torch.float64 and theta.is_contiguous() and theta.shape == (self.S, NPARAM)
        cov = torch.empty(self.S, NPARAM, NPARAM, dtype=torch.float64, device=theta.device)
        ok = torch.empty(self.S, dtype=torch.int32, device=theta.device)
        _check(lib().celeste_covariance_batch(self.handle, _ptr(theta), _ptr(cov), _ptr(ok), _stream(stream)))
        return cov, ok

    def extract_patches(self, stream=None):
        """The warm-start network's input for every source: int16 [S, 32, 32, 5] BF16 bit patterns."""
        x = torch.empty(self.S, 32, 32, 5, dtype=torch.int16, device=self.device)
        _check(lib().celeste_extract_patches(self.handle, _ptr(x), _stream(stream)))
        return x

    def refresh_pixels(self, stream=None):
        """New counts in the same device images: re-gather the patch pixels (layout unchanged)."""
        _check(lib().celeste_problem_refresh_pixels(self.handle, _stream(stream)))

    def rebind(self, stream=None):
        """Upload the layout again and re-gather the patch pixels from the device images."""
        _check(lib().celeste_problem_bind(self.handle, self._ws_ptr, ctypes.c_size_t(self._ws_bytes), _stream(stream)))

    def profile_start(self):
        _check(lib().celeste_profile_start(self.handle))

    def profile_stop(self):
        st = ProfileStats()
        _check(lib().celeste_profile_stop(self.handle, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in ProfileStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib().celeste_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tr_solve_batch(B, g, delta, warps=1, lam_hint=None, return_lambda=False, stream=None):
    """Trust-region subproblems on the device: B [n,27,27], g [n,27], delta [n] float64 CUDA tensors, solved
    on one warp or one four-warp CTA per problem (warps 1 or 4), the multiplier search optionally placed
    around lam_hint [n].  Returns (p [n,27], pred [n], hard [n] int32) and, with return_lambda, the
    multipliers [n]."""
    n = g.shape[0]
    for t in (B, g, delta) + ((lam_hint,) if lam_hint is not None else ()):
        assert t.dtype == torch.float64 and t.is_contiguous() and t.is_cuda
    p = torch.empty(n, NPARAM, dtype=torch.float64, device=g.device)
    pred = torch.empty(n, dtype=torch.float64, device=g.device)
    hard = torch.empty(n, dtype=torch.int32, device=g.device)
    lam = torch.empty(n, dtype=torch.float64, device=g.device)
    if warps == 1 and lam_hint is None and not return_lambda:
        _check(lib().celeste_tr_solve_batch(_ptr(B), _ptr(g), _ptr(delta), ctypes.c_int(n), _ptr(p), _ptr(pred),
                                            _ptr(hard), _stream(stream)))
    else:
        _check(lib().celeste_tr_solve_batch_ex(_ptr(B), _ptr(g), _ptr(delta), ctypes.c_int(n), ctypes.c_int(warps),
                                               _ptr(lam_hint) if lam_hint is not None else None, _ptr(p), _ptr(pred),
                                               _ptr(hard), _ptr(lam), _stream(stream)))
    return (p, pred, hard, lam) if return_lambda else (p, pred, hard)


def tr_reciprocal(x, stream=None):
    """The subproblem solver's float64 reciprocal applied to a float64 CUDA tensor (for its error test)."""
    assert x.dtype == torch.float64 and x.is_contiguous() and x.is_cuda
    r = torch.empty_like(x)
    _check(lib().celeste_tr_reciprocal(_ptr(x), _ptr(r), ctypes.c_int(x.numel()), _stream(stream)))
    return r


def measure_peak(kind, stream=None):
    """Measured rate of one pipe of the current device: kind "fp32" (FMA flop/s), "ex2" (special-function
    exponentials/s), "fp64" (FMA flop/s) or "fp32x2" (packed two-wide FP32 FMA flop/s).  Returns (rate,
    seconds of the timed launch)."""
    k = {"fp32": 0, "ex2": 1, "fp64": 2, "fp32x2": 3}[kind]
    rate, sec = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib().celeste_measure_peak(ctypes.c_int(k), ctypes.byref(rate), ctypes.byref(sec), _stream(stream)))
    return rate.value, sec.value


def _joint_pairs(handle):
    n = ctypes.c_int64(0)
    _check(lib().celeste_joint_pairs(handle, None, ctypes.c_int64(0), ctypes.byref(n)))
    out = np.zeros((max(n.value, 1), 2), dtype=np.int32)
    _check(lib().celeste_joint_pairs(handle, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(n.value),
                                     ctypes.byref(n)))
    return out[:n.value]


class HostProblem:
    """Layout-only handle (no device memory): validation and counts, usable without a GPU."""

    def __init__(self, scene, tile_pixels=256, hessian_mode=0):
        L = lib()
        n = len(scene.images)
        self._imgs = (ImageDesc * n)()
        for k, im in enumerate(scene.images):
            d = self._imgs[k]
            d.height, d.width = im.pixels.shape
            d.band = int(im.band)
            d.pixels = 1          # never dereferenced on the host
            d.sky, d.iota = float(im.sky), float(im.iota)
            d.wcs[:] = [float(v) for v in im.wcs]
            d.psf[:] = [float(v) for v in np.asarray(im.psf, np.float64).reshape(-1)]
        self._u0 = np.ascontiguousarray(scene.u0, np.float64)
        self._rad = np.ascontiguousarray(scene.radius, np.int32)
        desc = ProblemDesc()
        desc.n_images = n
        desc.images = self._imgs
        desc.n_sources = self._u0.shape[0]
        desc.u0 = self._u0.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        desc.radius = self._rad.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        desc.priors[:] = [float(v) for v in scene.priors]
        desc.exp_nu[:] = [float(v) for v in scene.exp_nu]
        desc.exp_tau[:] = [float(v) for v in scene.exp_tau]
        desc.dev_nu[:] = [float(v) for v in scene.dev_nu]
        desc.dev_tau[:] = [float(v) for v in scene.dev_tau]
        desc.tile_pixels = int(tile_pixels)
        desc.hessian_mode = int(hessian_mode)
        self.desc = desc
        h = ctypes.c_void_p()
        _check(L.celeste_problem_create(ctypes.byref(desc), ctypes.byref(h)))
        self.handle = h

    def counts(self):
        c = (ctypes.c_int64 * 5)()
        _check(lib().celeste_problem_counts(self.handle, c))
        return dict(sources=c[0], patches=c[1], tiles=c[2], pixels=c[3], neighbours=c[4])

    def workspace_bytes(self):
        return lib().celeste_problem_workspace_bytes(self.handle)

    def joint_pairs(self):
        """[n_pairs, 2] int32: source pairs s < t whose windows overlap (host only)."""
        return _joint_pairs(self.handle)

    def __del__(self):
        try:
            lib().celeste_problem_destroy(self.handle)
        except Exception:
            pass
