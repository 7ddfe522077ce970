"""Oracle of the Herschel-Bulkley fit sigma = sigma_Y + A S^beta (the law the
paper fits to its flow curve, section "Numerical Results").

TEST INFRASTRUCTURE ONLY.  Plain definition: for each beta the best
(sigma_Y, A) is the ordinary least-squares solution of the linear model
[1, S^beta] (numpy.linalg.lstsq); beta minimises the residual sum of squares,
located on a uniform grid and refined with scipy's bounded scalar minimiser.
"""
import numpy as np
from scipy.optimize import minimize_scalar


def _rss(S, sig, beta):
    X = np.stack([np.ones_like(S), S ** beta], axis=1)
    coef, *_ = np.linalg.lstsq(X, sig, rcond=None)
    r = sig - X @ coef
    return float(r @ r), coef


def fit(S, sig, beta_lo=0.02, beta_hi=3.0, n_grid=20001):
    S = np.asarray(S, dtype=np.float64)
    sig = np.asarray(sig, dtype=np.float64)
    grid = np.linspace(beta_lo, beta_hi, n_grid)
    vals = [_rss(S, sig, b)[0] for b in grid]
    k = int(np.argmin(vals))
    lo, hi = grid[max(k - 1, 0)], grid[min(k + 1, n_grid - 1)]
    res = minimize_scalar(lambda b: _rss(S, sig, b)[0], bounds=(lo, hi), method="bounded",
                          options={"xatol": 1e-14})
    beta = float(res.x) if res.fun <= vals[k] else float(grid[k])
    rss, coef = _rss(S, sig, beta)
    return dict(sigma_y=float(coef[0]), A=float(coef[1]), beta=beta, rss=rss)
