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
