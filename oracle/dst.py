"""DST-I by its defining sum (oracle; test infrastructure).

X_k = sum_{j=1}^{n} x_j sin(pi j k / (n + 1)),  k = 1..n,

the transform that diagonalises the compact operators on zero-Dirichlet grid
functions (the sine expansions of Lemma 4 and its appendix proof).  Applying
it twice gives (n + 1)/2 times the identity (discrete sine orthogonality,
appendix: h sum_j sin(k pi j/N) sin(l pi j/N) = delta_kl / 2).
"""

import numpy as np


def sine_matrix(n: int) -> np.ndarray:
    j = np.arange(1, n + 1)
    return np.sin(np.pi * np.outer(j, j) / (n + 1))


def dst1(x: np.ndarray, axis: int = -1) -> np.ndarray:
    """DST-I of ``x`` along ``axis`` (numpy axis numbering), by matrix product."""
    x = np.asarray(x, dtype=np.float64)
    S = sine_matrix(x.shape[axis])
    return np.moveaxis(np.tensordot(S, np.moveaxis(x, axis, 0), axes=(1, 0)), 0, axis)
