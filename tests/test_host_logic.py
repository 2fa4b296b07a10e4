"""Host-side logic of the Python layer, on CPU: the warm-start assembly and the block-coordinate
orchestration (against a stand-in problem that records its calls)."""
import numpy as np
import torch

from paper_1611_03404_gb300 import NBR_FULL, NBR_WINDOW, WANT_GRAD
from paper_1611_03404_gb300.blockcoord import block_coordinate
from paper_1611_03404_gb300.cnn import NET_PARAMS, training_targets, warm_start


def test_warm_start_takes_only_the_listed_parameters():
    rng = np.random.default_rng(0)
    cat = torch.as_tensor(rng.standard_normal((5, 27)))
    pred = torch.as_tensor(rng.standard_normal((5, 27)))
    th = warm_start(cat, pred)
    for j in range(27):
        if j in NET_PARAMS:
            assert torch.equal(th[:, j], pred[:, j] + (cat[:, j] if j < 2 else 0.0))
        else:
            assert torch.equal(th[:, j], cat[:, j])
    # a predicted position is an offset from the catalog position
    th2 = warm_start(cat, pred, params=[0, 1])
    assert torch.allclose(th2[:, 0:2], cat[:, 0:2] + pred[:, 0:2])
    assert torch.equal(th2[:, 2:], cat[:, 2:])


def test_training_targets_are_offsets_in_position():
    rng = np.random.default_rng(1)
    th = torch.as_tensor(rng.standard_normal((4, 27)))
    u0 = torch.as_tensor(rng.standard_normal((4, 2)))
    t = training_targets(th, u0)
    assert torch.allclose(t[:, 0:2], th[:, 0:2] - u0)
    assert torch.equal(t[:, 2:], th[:, 2:])


class _StandIn:
    """Records the calls block_coordinate makes; each Newton call moves every source halfway
    towards a fixed target and reports convergence."""

    def __init__(self, S, target):
        self.S, self.target, self.calls = S, target, []

    def render_background(self, nbr_theta, mode=NBR_FULL):
        self.calls.append(("background", mode, nbr_theta.clone()))

    def newton_batch(self, theta, **opts):
        self.calls.append(("newton", opts))
        theta += 0.5 * (self.target - theta)
        S = theta.shape[0]
        return (torch.ones(S, dtype=torch.float64), torch.full((S,), 3, dtype=torch.int32),
                torch.zeros(S, dtype=torch.int32), torch.zeros(S, dtype=torch.float64))

    def elbo_batch(self, theta, want):
        assert want == WANT_GRAD
        self.calls.append(("grad",))
        return None, self.target - theta, None


def test_block_coordinate_passes_and_residual():
    S = 6
    rng = np.random.default_rng(2)
    target = torch.as_tensor(rng.standard_normal((S, 27)))
    theta0 = torch.zeros(S, 27, dtype=torch.float64)
    prob = _StandIn(S, target)
    theta, hist = block_coordinate(prob, theta0, passes=3, mode=NBR_WINDOW, residual=True, max_iter=7)
    # every pass renders the neighbours at the previous pass's result in the requested mode,
    # runs Newton with the given options, then (residual) re-renders at the result for the gradient
    kinds = [c[0] for c in prob.calls]
    assert kinds == ["background", "newton", "background", "grad"] * 3
    backgrounds = [c for c in prob.calls if c[0] == "background"]
    assert all(c[1] == NBR_WINDOW for c in backgrounds)
    assert torch.equal(backgrounds[0][2], theta0)
    assert all(c[1] == {"max_iter": 7} for c in prob.calls if c[0] == "newton")
    assert torch.allclose(theta, target * (1 - 0.5 ** 3))
    for k, h in enumerate(hist):
        gap = (target * 0.5 ** (k + 1)).abs()
        assert np.isclose(h["grad_max"], float(gap.max())) and np.isclose(h["grad_median"], float(gap.max(1).values.median()))
        assert h["converged"] == S and h["newton_iters_mean"] == 3.0
    assert hist[0]["max_change"] > hist[1]["max_change"] > hist[2]["max_change"]


def test_clock_summary_reads_throttle_reasons():
    import bench
    cs = bench.ClockSampler(0)
    assert cs.summary()["reasons"] == ["unsampled"]
    na, act = "Not Active", "Active"
    cs.rows = [["2070", "2070", "900.1", na, na, na, na],
               ["1980", "2070", "1401.0", na, na, na, act],
               ["2070", "2070", "1350.7", na, na, na, na]]
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    cs.rows.append(["1410", "2070", "700.0", act, na, act, na])
    assert bench.ClockSampler.summary(cs)["reasons"] == ["hw_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


def test_bench_subscene_keeps_the_oracle_objective():
    """The CPU baseline times the oracle on a sub-scene per sampled source (the source, every source
    whose patch can overlap one of its patches, the images holding its patch centre); the source's
    objective there is the one on the whole scene: same patches, same neighbours, same ELBO."""
    import bench
    import synth
    from oracle import celeste_oracle as O
    sc = synth.tiny(seed=31, n_sources=14, n_images=3, H=90, W=100, radius=(4, 12))
    full = O.Oracle(sc)
    for s in (0, 5, 9):
        sub = bench.subscene(sc, s)
        orc = O.Oracle(sub)
        assert [r[1:] for r in orc.rects[0]] == [r[1:] for r in full.rects[s]]
        mapped = {int(np.nonzero((sc.u0 == sub.u0[t]).all(1))[0][0]) for lst in orc.nbr[0].values() for t in lst}
        assert mapped == {t for lst in full.nbr[s].values() for t in lst}
        if full.rects[s]:
            assert orc.elbo(0, sub.theta0[0], sub.theta0) == full.elbo(s, sc.theta0[s], sc.theta0)


def test_bench_parses_the_driver_command_line():
    import bench
    a = bench.parse(["--gpus", "1", "--steps", "20", "--warmup", "5"])
    assert a.workload == "mosaic" and a.hessian == "auto" and a.tile == 0 and a.warm_start
    assert bench.workload_config(a)["workload"] == "mosaic_10x10_fields_100000src"
    # the reference arm prints the same config as the GPU arm
    b = bench.parse(["--impl", "reference", "--steps", "20", "--warmup", "5"])
    assert bench.workload_config(a) == bench.workload_config(b)


def test_bench_patch_pixel_count_matches_the_library_layout():
    import bench
    import synth
    import paper_1611_03404_gb300 as P
    import __graft_entry__
    __graft_entry__.build()
    for seed in (3, 4):
        sc = synth.tiny(seed=seed, n_sources=30, n_images=3, H=80, W=90, radius=(3, 20))
        c = P.HostProblem(sc, tile_pixels=128).counts()
        assert bench.mean_patch_pixels(sc, chunk=7) == c["pixels"] / c["sources"]
