"""Matrix-free application of the coupled HOC equations (oracle; test infrastructure).

Given full-grid U and V (V on the faces holding Q), evaluate the three block
rows of the coupled system of Sec. 2.2 by array slicing:
    r_u = L_h U - M(V / alpha)                    at interior points
    r_v = -L_h V - M f                            at interior points
    r_q = alpha_p (delta_nn U + lapt_gD) - Q_p    at face points (Lemma 1's R)
This is a second, independent statement of the same equations as
``coupled.assemble`` (slices instead of sparse rows) and serves as a residual
certificate on grids too large for a direct solve.
"""

from __future__ import annotations

import numpy as np

from .stencils import laplacian, one_sided_weights, weighting


def _shift(A, off):
    """View of A over interior points shifted by ``off`` (offsets in axis order x, y, z)."""
    d = A.ndim
    sl = []
    for ax in range(d):
        a = d - 1 - ax          # numpy axis ax holds grid axis a
        o = off[a]
        n = A.shape[ax]
        sl.append(slice(1 + o, n - 1 + o))
    return A[tuple(sl)]


def apply_stencil(A, coeffs):
    out = None
    for off, c in coeffs.items():
        t = c * _shift(A, off)
        out = t if out is None else out + t
    return out


def face_trace(A, axis, side):
    """Values of a full-grid array on the relative interior of a face, in Q order."""
    d = A.ndim
    sl = [slice(1, -1)] * d
    sl[d - 1 - axis] = 0 if side == 0 else -1
    return A[tuple(sl)].reshape(-1)


def layer(A, axis, side, m):
    """Values m steps inward from a face, at the face's relative-interior positions."""
    d = A.ndim
    sl = [slice(1, -1)] * d
    n = A.shape[d - 1 - axis]
    sl[d - 1 - axis] = m if side == 0 else n - 1 - m
    return A[tuple(sl)].reshape(-1)


def coupled_residual(U, V, data):
    """Residuals (r_u, r_v, r_q) of the coupled equations for full-grid U, V."""
    N = list(data["N"])
    lo, hi = data["lo"], data["hi"]
    d = len(N)
    h = [(hi[a] - lo[a]) / N[a] for a in range(d)]
    alpha = np.asarray(data["alpha"], dtype=float)
    f = np.asarray(data["f"], dtype=float)
    L = laplacian(h)
    Mw = weighting(d)
    r_u = apply_stencil(U, L) - apply_stencil(V / alpha, Mw)
    r_v = -apply_stencil(V, L) - apply_stencil(f, Mw)
    gN = np.asarray(data["g_N"], dtype=float)
    lapt = np.asarray(data["lapt_gD"], dtype=float)
    r_q = []
    off = 0
    for a in range(d):
        (w0, w1, w2, w3), wg = one_sided_weights(h[a])
        for side in (0, 1):
            Q = face_trace(V, a, side)
            n = Q.size
            dnn = (w0 * face_trace(U, a, side) + w1 * layer(U, a, side, 1)
                   + w2 * layer(U, a, side, 2) + w3 * layer(U, a, side, 3) + wg * gN[off:off + n])
            r_q.append(face_trace(alpha, a, side) * (dnn + lapt[off:off + n]) - Q)
            off += n
    return r_u, r_v, np.concatenate(r_q)
