"""Compact fourth-order stencils of the augmented HOC scheme (oracle; test infrastructure).

Each stencil is returned as a dict {offset tuple: coefficient}; offsets are
ordered (dx, dy[, dz]).  h is the per-axis mesh spacing.

Sources and readings:
  * 3D Laplacian L_h: the 19-point operator printed in Sec. 2.2 as the planes
    L_{k-1}, L_k, L_{k+1}.  The printed prefactor 1/2 is read as 1/12 (with
    1/2 the operator is six times too large and is not consistent with the
    weighting M = (1/12)[...] printed beside it); with 1/12 it reproduces the
    Laplacian to fourth order, L_h p = M(Lap p) exactly for every polynomial of
    total degree <= 5 (pinned in the tests).
  * 2D Laplacian: Sec. 3.1 prints a five-point-looking operator; it is read as
    the nine-point compact operator with corner weight (1/h_x^2 + 1/h_y^2)/12,
    edge weights (10/h_a^2 - 2/h_b^2)/12 and centre -20(1/h_x^2 + 1/h_y^2)/12.
    Only this operator yields the recurrence of the 2D proof of Lemma 4 in the
    appendix, (4 + 2cos t) c(i-1) + (8cos t - 20) c(i) + (4 + 2cos t) c(i+1) = 0
    for h_x = h_y (pinned in the tests), and it is degree-5 exact.
  * Weighting M: (1/12)[1; 8; 1] cross in 2D (Sec. 3.1), (1/12)[6 centre, 1 per
    face] in 3D (Sec. 2.2).
  * One-sided second normal derivative at a clamped face (Sec. 2.2):
      u_nn ~ h^-2 (-85/18 U0 + 6 U1 - 3/2 U2 + 2/9 U3) + 11/(3h) g_N,
    with U_m the value m steps inward along the normal, h the spacing along
    the normal and g_N the outward normal derivative; the same coefficients
    hold on every face ("analogous formulas", Sec. 2.2).
"""

from __future__ import annotations

from fractions import Fraction
from typing import Dict, Sequence, Tuple

ONE_SIDED = (Fraction(-85, 18), Fraction(6), Fraction(-3, 2), Fraction(2, 9))
ONE_SIDED_GN = Fraction(11, 3)


def laplacian(h: Sequence[float]) -> Dict[Tuple[int, ...], float]:
    """The compact fourth-order Laplacian L_h (2D: 9 points, 3D: 19 points)."""
    d = len(h)
    inv = [1.0 / (hh * hh) for hh in h]
    c: Dict[Tuple[int, ...], float] = {}
    if d == 2:
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dx and dy:
                    v = inv[0] + inv[1]
                elif dx:
                    v = 10 * inv[0] - 2 * inv[1]
                elif dy:
                    v = 10 * inv[1] - 2 * inv[0]
                else:
                    v = -20 * (inv[0] + inv[1])
                c[(dx, dy)] = v / 12.0
        return c
    if d == 3:
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    o = (dx, dy, dz)
                    nz = [a for a in range(3) if o[a] != 0]
                    if len(nz) == 3:
                        continue  # the 19-point operator has no cube-corner entries
                    if len(nz) == 2:
                        v = inv[nz[0]] + inv[nz[1]]
                    elif len(nz) == 1:
                        a = nz[0]
                        v = 8 * inv[a] - 2 * sum(inv[b] for b in range(3) if b != a)
                    else:
                        v = -16 * sum(inv)
                    c[o] = v / 12.0
        return c
    raise ValueError("dim must be 2 or 3")


def weighting(d: int) -> Dict[Tuple[int, ...], float]:
    """The weighting operator M applied to right-hand sides."""
    c: Dict[Tuple[int, ...], float] = {}
    zero = (0,) * d
    c[zero] = (8.0 if d == 2 else 6.0) / 12.0
    for a in range(d):
        for s in (-1, 1):
            o = [0] * d
            o[a] = s
            c[tuple(o)] = 1.0 / 12.0
    return c


def one_sided_weights(h_n: float):
    """Weights (w0, w1, w2, w3) on U0..U3 and the weight on g_N of u_nn."""
    w = tuple(float(x) / (h_n * h_n) for x in ONE_SIDED)
    return w, float(ONE_SIDED_GN) / h_n
