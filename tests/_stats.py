"""Small statistics helpers for the statistical pins (no method arithmetic)."""
import numpy as np


def blocking_error(x) -> float:
    """Standard error of the mean of a correlated series by Flyvbjerg-Petersen
    blocking (J. Chem. Phys. 91, 461 (1989)): halve the series repeatedly and
    take the largest naive error over the levels that keep >= 32 blocks."""
    x = np.asarray(x, np.float64)
    best = 0.0
    while x.size >= 32:
        n = x.size
        err = np.sqrt(np.var(x, ddof=1) / n) if n > 1 else 0.0
        best = max(best, err)
        x = 0.5 * (x[: n // 2 * 2 : 2] + x[1 : n // 2 * 2 : 2])
    return float(best)


def langevin(x: float) -> float:
    """L(x) = coth(x) - 1/x."""
    return 1.0 / np.tanh(x) - 1.0 / x


def t3(dof: int) -> float:
    """The bound, in standard errors, with the two-sided coverage of 3 sigma
    of a normal law (99.73%) when the standard error itself is estimated
    from `dof` degrees of freedom: the Student-t quantile.  It tends to 3 as
    dof grows (3.96 at 10, 3.27 at 30)."""
    from scipy import stats
    return float(stats.t.ppf(1.0 - 0.0026997960632601866 / 2.0, dof))


def diff_within_t3(a, b):
    """(difference of the means of two sets of independent run means, its
    standard error from the pooled spread, the 3-sigma-equivalent bound)."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    se = float(np.sqrt(a.var(ddof=1) / a.size + b.var(ddof=1) / b.size))
    return float(a.mean() - b.mean()), se, t3(a.size + b.size - 2) * se
