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
