"""C ABI checks that need no GPU: the library loads, exports every declared entry point, validates
descriptors, and lays out patches / neighbours / tiles exactly as the oracle defines them."""
import os
import re

import numpy as np
import pytest

import synth
from oracle import celeste_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1611_03404_gb300 as P
    return P


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"\b(celeste_[a-z_]+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(pkg):
    lib = pkg.lib()
    declared = _declared_symbols()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name


def test_strerror_codes(pkg):
    lib = pkg.lib()
    assert lib.celeste_strerror(0) == b"ok"
    assert lib.celeste_strerror(1) == b"invalid argument"
    assert lib.celeste_strerror(999) == b"unknown error"


def _layout_reference(scene, tile):
    rects = O.patch_rects(scene)
    nbr = O.neighbour_lists(scene, rects)
    patches = sum(len(r) for r in rects)
    pixels = sum((x1 - x0 + 1) * (y1 - y0 + 1) for r in rects for (_, x0, x1, y0, y1) in r)
    tiles = sum(-(-((x1 - x0 + 1) * (y1 - y0 + 1)) // tile) for r in rects for (_, x0, x1, y0, y1) in r)
    nb = sum(len(v) for d in nbr for v in d.values())
    return dict(sources=scene.n_sources, patches=patches, tiles=tiles, pixels=pixels, neighbours=nb)


@pytest.mark.parametrize("seed", [3, 4, 5])
@pytest.mark.parametrize("tile", [128, 256, 1024])
def test_layout_matches_oracle_geometry(pkg, seed, tile):
    sc = synth.tiny(seed=seed, n_sources=6, n_images=3, H=40, W=44, radius=(3, 12))
    hp = pkg.HostProblem(sc, tile_pixels=tile)
    assert hp.counts() == _layout_reference(sc, tile)
    assert hp.workspace_bytes() > 0


def test_layout_edge_sources(pkg):
    """Sources at the image corners and outside some images: clipped or absent patches."""
    sc = synth.tiny(seed=9, n_sources=4, n_images=2, H=30, W=30, radius=(5, 5))
    sc.u0 = np.array([[0.2, 0.1], [29.4, 29.3], [-3.0, 15.0], [15.0, 15.0]])
    hp = pkg.HostProblem(sc)
    assert hp.counts() == _layout_reference(sc, 256)


def _expect_invalid(pkg, sc, **kw):
    with pytest.raises(pkg.CelesteError, match="invalid argument"):
        pkg.HostProblem(sc, **kw)


def test_validation_rejects_bad_descriptors(pkg):
    base = lambda: synth.tiny(seed=1, n_sources=2, n_images=2)
    sc = base()
    sc.images[0].sky = float("nan")
    _expect_invalid(pkg, sc)
    sc = base()
    sc.images[1].iota = -1.0
    _expect_invalid(pkg, sc)
    sc = base()
    sc.radius = np.array([0, 5], np.int32)
    _expect_invalid(pkg, sc)
    sc = base()
    sc.radius = np.array([65, 5], np.int32)
    _expect_invalid(pkg, sc)
    sc = base()
    sc.u0 = sc.u0.copy()
    sc.u0[0, 0] = np.inf
    _expect_invalid(pkg, sc)
    sc = base()
    sc.exp_nu = sc.exp_nu * 1.1
    _expect_invalid(pkg, sc)
    sc = base()
    sc.images[0].wcs = np.array([1.0, 0.0, 2.0, 0.0, 0.0, 0.0])
    _expect_invalid(pkg, sc)
    sc = base()
    sc.images[0].psf = sc.images[0].psf.copy()
    sc.images[0].psf[0, 3, 0] = 9.0
    _expect_invalid(pkg, sc)
    sc = base()
    sc.images[0].band = 7
    _expect_invalid(pkg, sc)
    sc = base()
    sc.priors = np.array([1.5, 2.0, 1.0, 0.0, 0.25])
    _expect_invalid(pkg, sc)
    _expect_invalid(pkg, base(), tile_pixels=100)


def test_hessian_mode_validation(pkg):
    """The tensor-core SYRK modes exist for 128-pixel tiles only; unknown modes are refused."""
    sc = synth.tiny(seed=1, n_sources=2, n_images=2)
    for mode in (pkg.HESS_FP32, pkg.HESS_TF32, pkg.HESS_BF16X3, pkg.HESS_BF16X6, pkg.HESS_TF32X3):
        assert pkg.HostProblem(sc, tile_pixels=128, hessian_mode=mode).counts()["sources"] == 2
    for mode, tile in ((5, 128), (-1, 128), (pkg.HESS_TF32, 256), (pkg.HESS_BF16X3, 512), (pkg.HESS_BF16X6, 256),
                       (pkg.HESS_TF32X3, 1024)):
        with pytest.raises(pkg.CelesteError, match="invalid argument"):
            pkg.HostProblem(sc, tile_pixels=tile, hessian_mode=mode)


@pytest.mark.parametrize("seed,kw", [(11, dict(n_sources=3, n_images=3)),
                                     (3, dict(n_sources=5, n_images=2, H=40, W=44, radius=(6, 12))),
                                     (21, dict(n_sources=8, n_images=3, H=60, W=64, radius=(3, 12)))])
def test_joint_pairs_match_the_oracle_geometry(pkg, seed, kw):
    """The library's overlapping source pairs (host layout, no GPU) equal the oracle's."""
    from oracle import celeste_oracle as O
    from oracle import joint_oracle as JO
    sc = synth.tiny(seed=seed, **kw)
    got = [tuple(int(v) for v in p) for p in pkg.HostProblem(sc, tile_pixels=128).joint_pairs()]
    assert got == JO.overlapping_pairs(O.Oracle(sc))


def test_joint_pairs_on_a_field(pkg):
    from oracle import celeste_oracle as O
    from oracle import joint_oracle as JO
    sc = synth.field(seed=1622, W=768, H=560, n_sources=200)
    got = [tuple(int(v) for v in p) for p in pkg.HostProblem(sc, tile_pixels=128).joint_pairs()]
    ref = JO.overlapping_pairs(O.Oracle(sc))
    assert got == ref and len(ref) > 20


def test_joint_pairs_empty_when_no_window_overlaps(pkg):
    sc = synth.tiny(seed=11, n_sources=3, n_images=3)
    sc.radius = np.full_like(sc.radius, 1)
    assert len(pkg.HostProblem(sc, tile_pixels=128).joint_pairs()) == 0


def test_joint_workspace_is_caller_bound(pkg):
    """The joint calls' memory is a caller-bound workspace: its size is known on the host, and binding
    needs a bound problem (no device memory is touched here)."""
    import ctypes
    sc = synth.tiny(seed=3, n_sources=5, n_images=2, H=40, W=44, radius=(6, 12))
    hp = pkg.HostProblem(sc, tile_pixels=128)
    L = pkg.lib()
    n = L.celeste_joint_workspace_bytes(hp.handle)
    assert n > 0 and n % 256 == 0
    assert L.celeste_joint_workspace_bytes(None) == 0
    rc = L.celeste_joint_bind(hp.handle, ctypes.c_void_p(256), ctypes.c_size_t(n), None)
    assert rc == 5 and "bind the problem" in L.celeste_last_error_detail().decode()
