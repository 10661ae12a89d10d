"""MuyGPs hyperparameter training (Algorithm 1): minimise the LOOCV objective
Q(theta) of Eq. 5 over a batch, with each evaluation on the GPU through
fmgp_loocv_objective and the outer loop by L-BFGS-B (the optimiser the paper
names) on log-parameters with finite-difference gradients.

The neighbour table does not depend on theta (the kernels are isotropic and
rank by distance), so it is built once and reused for every evaluation."""
import math

import numpy as np
import torch

from . import _binding as fb

_PARAMS = ("length_scale", "nugget", "variance")


def optimize_hyperparameters(X, Y, batch, k, kernel, params=("length_scale",), bounds=None,
                             precision=fb.PREC_MIXED, maxiter=50, nbr=None):
    """Returns a dict with the optimised kernel (an fmgp Kernel), the objective
    before and after, the number of objective evaluations and the history.

    X, Y, batch: CUDA tensors (n x d, n x r FP64, b int64); k: neighbours per
    batch point (excluding the point); kernel: starting fb.Kernel; params: the
    Kernel fields to optimise (length_scale, nugget, variance); bounds: dict
    field -> (lo, hi), defaults to generous ranges."""
    from scipy.optimize import minimize

    for p in params:
        if p not in _PARAMS:
            raise ValueError(f"cannot optimise {p!r}; choose from {_PARAMS}")
    if nbr is None:
        nbr, _ = fb.fmgp_build_knn(X, k)
    default_bounds = {"length_scale": (1e-4, 1e4), "nugget": (1e-10, 1.0),
                      "variance": (1e-6, 1e6)}
    bounds = dict(default_bounds, **(bounds or {}))
    x0 = np.array([math.log(getattr(kernel, p)) for p in params])
    lb = [math.log(bounds[p][0]) for p in params]
    ub = [math.log(bounds[p][1]) for p in params]
    history = []

    def make(x):
        kk = fb.Kernel(kernel.kind, kernel.nu, kernel.length_scale, kernel.variance, kernel.nugget)
        for p, v in zip(params, x):
            setattr(kk, p, float(math.exp(v)))
        return kk

    # the optimiser sees log Q: Q itself can be tiny (1e-4 and below), which
    # would put its gradient under L-BFGS-B's default tolerance at once
    def objective(x):
        q, _ = fb.fmgp_loocv_objective(X, Y, nbr, k, batch, make(x), precision,
                                       raise_on_not_spd=False)
        if not (math.isfinite(q) and q > 0):
            q = 1e300
        history.append((x.copy(), q))
        return math.log(q)

    q0 = math.exp(objective(x0))
    res = minimize(objective, x0, method="L-BFGS-B", bounds=list(zip(lb, ub)),
                   options={"maxiter": maxiter, "eps": 1e-5, "ftol": 1e-12, "gtol": 1e-8})
    best = make(res.x)
    return {"kernel": best, "q_start": q0, "q_best": float(math.exp(res.fun)),
            "evaluations": len(history),
            "theta": {p: float(math.exp(v)) for p, v in zip(params, res.x)},
            "converged": bool(res.success), "history": history}
