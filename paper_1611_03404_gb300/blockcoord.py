"""Block-coordinate passes (paper, Sec. "Variational Inference": each source is optimised with its
neighbours held fixed; repeating the sweep with the neighbours at their new values is block
coordinate ascent on the joint ELBO).  Orchestration only: every evaluation and Newton step runs
in the library's kernels.

With mode=NBR_WINDOW every source's light is counted on its own window only, so each per-source
objective has the joint objective's gradient with respect to that source (paper, concluding
section: a stationary point of the objective over all light sources jointly); the passes are
then block-coordinate ascent on that joint objective, and `residual` reports its gradient at the
end of each pass (the neighbours moved during the pass, so it is not zero until the sweep has
converged)."""
import torch

from .celeste import NBR_FULL, WANT_GRAD


def block_coordinate(prob, theta0, passes=2, mode=NBR_FULL, residual=False, radius_world=None, **newton_opts):
    """Runs `passes` sweeps: the first with the neighbours fixed at theta0 (the catalog), each later
    one with the neighbours at the previous sweep's result.  Returns the final parameters and, per
    pass, the largest and mean absolute parameter change, the largest position change, the mean
    Newton iteration count and the number of converged sources; with `residual`, also the largest
    and median over sources of max_i |dL/dtheta_i| at the pass's result with every neighbour at its
    new value (the joint objective's gradient when mode is NBR_WINDOW).  With radius_world (a tensor
    [S] of patch half-widths in world units) each pass also counts the sources whose position has
    moved further than that from theta0: their light has left the patch their objective covers."""
    theta = theta0.clone().contiguous()
    history = []
    for k in range(passes):
        prev = theta.clone()
        prob.render_background(prev, mode=mode)
        _, iters, status, elbo = prob.newton_batch(theta, **newton_opts)
        change = (theta - prev).abs()
        pos = change[:, 0:2].max(1).values
        history.append({"pass": k, "max_change": float(change.max()), "mean_change": float(change.mean()),
                         "max_position_change": float(pos.max()),
                         "p99_position_change": float(torch.quantile(pos, 0.99)),
                         "newton_iters_mean": float(iters.double().mean()),
                         "converged": int((status == 0).sum()),
                         "status_counts": [int((status == k).sum()) for k in range(4)],
                         "left_window": None if radius_world is None else
                         int(((theta[:, 0:2] - theta0[:, 0:2]).abs().max(1).values > radius_world).sum()),
                         "elbo_sum_finite": float(elbo[torch.isfinite(elbo)].sum()),
                         "nonfinite": int((~torch.isfinite(elbo)).sum())})
        if residual:
            prob.render_background(theta, mode=mode)
            _, g, _ = prob.elbo_batch(theta, want=WANT_GRAD)
            gm = g.abs().max(1).values
            history[-1]["grad_max"] = float(gm.max())
            history[-1]["grad_median"] = float(gm.median())
    return theta, history
