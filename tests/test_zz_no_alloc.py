"""celeste_elbo_batch_noalloc: the evaluation for callers that may not allocate device memory.

Such callers (a pre-sized memory arena, an allocator owned by another framework, a request path
that must not allocate) get one entry point whose kernel scratch lives in a fixed device array
inside the library.  These tests call it through the C ABI and check it against
celeste_elbo_batch, which uses the caller-provided workspace, with the tolerances of the parity
tests, on two calls in a row (the array keeps the previous call's contents).  The file is named
to be collected last.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import synth

ELBO_RTOL, GRAD_RTOL, HESS_RTOL, GRAD_FLOOR, HESS_FLOOR = 1e-6, 1e-4, 1e-4, 1e-3, 1e-2


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1611_03404_gb300 as P
    fn = P.lib().celeste_elbo_batch_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p] * 6
    return P


def _noalloc(P, handle, theta, S):
    dev = theta.device
    e = torch.full((S,), math.nan, dtype=torch.float64, device=dev)
    g = torch.full((S, 27), math.nan, dtype=torch.float64, device=dev)
    h = torch.full((S, 27, 27), math.nan, dtype=torch.float64, device=dev)
    rc = P.lib().celeste_elbo_batch_noalloc(handle, ctypes.c_void_p(theta.data_ptr()), ctypes.c_void_p(e.data_ptr()),
                                            ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(h.data_ptr()),
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, P.lib().celeste_last_error_detail().decode()
    torch.cuda.synchronize()
    return e.cpu().numpy(), g.cpu().numpy(), h.cpu().numpy()


def _close(got, ref):
    e, g, h = got
    E, G, H = ref
    for s in range(len(E)):
        assert abs(e[s] - E[s]) <= ELBO_RTOL * abs(E[s])
        gs = np.maximum(np.abs(G[s]), GRAD_FLOOR * np.abs(G[s]).max())
        assert np.all(np.abs(g[s] - G[s]) <= GRAD_RTOL * gs)
        d = np.sqrt(np.abs(np.outer(np.diag(H[s]), np.diag(H[s]))))
        hs = np.maximum(np.abs(H[s]), HESS_FLOOR * d)
        assert np.all(np.abs(h[s] - H[s]) <= HESS_RTOL * np.where(hs > 0, hs, 1.0))


@pytest.mark.gpu
def test_noalloc_matches_workspace_path_two_calls(pkg):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P = pkg
    dev = torch.device("cuda:0")
    sc = synth.tiny(seed=21, n_sources=4, n_images=3, H=36, W=40, radius=(6, 14))
    prob = P.Problem(sc, device=dev)
    th1 = torch.as_tensor(sc.theta0, device=dev).contiguous()
    prob.render_background(th1)
    th2 = th1.clone()
    th2[:, 6] += 0.4
    th2[:, 0:2] += 0.15
    for th in (th1, th2):   # two calls in a row on the shared array
        ref = [t.cpu().numpy() for t in prob.elbo_batch(th)]
        torch.cuda.synchronize()
        _close(_noalloc(P, prob.handle, th, sc.n_sources), ref)
    # a second, differently sized problem reuses the same array
    sc2 = synth.single_source(seed=1611, size=41)
    prob2 = P.Problem(sc2, device=dev, tile_pixels=128)
    t2 = torch.as_tensor(sc2.theta0, device=dev).contiguous()
    prob2.render_background(t2)
    ref2 = [t.cpu().numpy() for t in prob2.elbo_batch(t2)]
    torch.cuda.synchronize()
    _close(_noalloc(P, prob2.handle, t2, sc2.n_sources), ref2)


def test_noalloc_rejects_problems_beyond_the_fixed_array(pkg):
    """A layout needing more scratch than the fixed array is refused before any device work."""
    P = pkg
    sc = synth.tiny(seed=2, n_sources=200, n_images=1, H=400, W=400, radius=(64, 64), noise=False)
    hp = P.HostProblem(sc, tile_pixels=128)
    c = hp.counts()
    need = (c["tiles"] * 436 + c["patches"] * 8228 + c["pixels"] * 8 + c["sources"] * 348)
    assert need > (8 << 20)
    z = ctypes.c_void_p(8)
    rc = P.lib().celeste_elbo_batch_noalloc(hp.handle, z, z, z, z, None)
    assert rc == 1
    assert "fixed array" in P.lib().celeste_last_error_detail().decode()
