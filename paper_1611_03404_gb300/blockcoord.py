"""Block-coordinate passes (paper, Sec. "Variational Inference": each source is optimised with its
neighbours held fixed; repeating the sweep with the neighbours at their new values is block
coordinate ascent on the joint ELBO).  Orchestration only: every evaluation and Newton step runs
in the library's kernels."""
import torch


def block_coordinate(prob, theta0, passes=2, **newton_opts):
    """Runs `passes` sweeps: the first with the neighbours fixed at theta0 (the catalog), each later
    one with the neighbours at the previous sweep's result.  Returns the final parameters and, per
    pass, the largest and mean absolute parameter change, the largest position change, the mean
    Newton iteration count and the number of converged sources."""
    theta = theta0.clone().contiguous()
    history = []
    for k in range(passes):
        prev = theta.clone()
        prob.render_background(prev)
        _, iters, status, elbo = prob.newton_batch(theta, **newton_opts)
        change = (theta - prev).abs()
        pos = change[:, 0:2].max(1).values
        history.append({"pass": k, "max_change": float(change.max()), "mean_change": float(change.mean()),
                         "max_position_change": float(pos.max()),
                         "p99_position_change": float(torch.quantile(pos, 0.99)),
                         "newton_iters_mean": float(iters.double().mean()),
                         "converged": int((status == 0).sum()), "elbo_sum": float(elbo.sum())})
    return theta, history
