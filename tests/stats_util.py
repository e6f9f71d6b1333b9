"""Statistical acceptance bands shared by the Monte Carlo tests.

An estimate A of a cell probability p from N walks has sd sqrt(p (1-p) / N).
The paper's estimator also carries the eps-shell bias beta(eps).  With many
entries a flat 4-sigma band fails by chance, so a matrix passes when

* every entry is within z_B sd + beta, z_B the Bonferroni-corrected two-sided
  normal quantile at family level alpha, and
* the number of entries outside 4 sd + beta is within the 1 - alpha quantile
  of Binomial(n_entries, P(|Z| > 4)).
"""
import math

import numpy as np
from scipy import stats

P4 = 2 * stats.norm.sf(4.0)


def beta_eps(eps, rho_max):
    """eps-shell bias bound: 2 (2/pi) rho_max eps (1 + ln(1/eps))."""
    return 2 * (2 / math.pi) * rho_max * eps * (1 + math.log(1 / eps))


def check_band(A, P, N, beta=0.0, alpha=1e-4):
    A = np.asarray(A, float)
    P = np.asarray(P, float)
    sd = np.sqrt(np.maximum(P * (1 - P), 1.0 / N) / N)
    n = A.size
    zb = stats.norm.isf(alpha / (2 * n))
    dev = np.abs(A - P)
    worst = float(np.max((dev - beta) / sd))
    out4 = int(np.sum(dev > 4 * sd + beta))
    allowed = int(stats.binom.isf(alpha, n, P4))
    ok = worst <= zb and out4 <= allowed
    return ok, dict(worst_z=worst, z_bonferroni=zb, outside_4sd=out4, allowed=allowed)
