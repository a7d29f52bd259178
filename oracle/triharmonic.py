"""The triharmonic mixed system, assembled and solved directly (oracle; test infrastructure).

Problem (the paper's triharmonic extension, Sec. 4.2 "Triharmonic equation",
Table 5): Lap^3 u = f in a box, with u, u_n and u_nn given on the clamped
faces and u, Lap u and Lap^2 u given on the other faces.  The mixed form
Lap u = v, Lap v = w, Lap w = f is discretised with the compact fourth-order
scheme of Sec. 2.2 (constant coefficient: L_h X = M(Lap x) for each
equation); v is data on the whole boundary (on a clamped face Lap u = u_nn +
Lap_t u is given); w is data on the other faces and on every edge and corner,
and on the relative interior of a clamped face it is the augmented unknown
q = w = Lap^2 u.

Unknowns: (U_p, V_p, W_p) interleaved per interior point, then Q on every
face point in the face layout of the library (x-, x+, y-, y+[, z-, z+]).
Equations, one block row each:
  (i)   L_h U - M V = 0     boundary U = g_D, boundary V = Lap u (data)
  (ii)  L_h V - M W = 0     boundary V data; W on a face point is Q
  (iii) L_h W = M f         W on a face point is Q, on edges and corners data
  (iv)  clamped face point p (normal axis a):
            Lap^2 u = u_ssss + 2 Lap_t u_ss + Lap_t^2 u  at p,
        with s the inward normal coordinate, u_ssss one-sided (below),
        u_ss = g_NN and the tangential terms data (lapt_w):
            delta4(U)_p + lapt_w_p - Q_p = 0;
        other faces: Lap^2 u is data there, the row is bilap_p - Q_p = 0.

Reading (the paper gives no formula for q): u_ssss at the face is
approximated one-sidedly the way Sec. 2.2 obtains its u_nn formula, by
undetermined coefficients on U_0 = g_D, U_1..U_4 and the known derivatives
u_s = -g_N and u_ss = g_NN:
    u_ssss ~ h^-4 sum_{m=0}^{4} c_m U_m + c_s h^-3 u_s + c_ss h^-2 u_ss,
exact for polynomials of degree <= 6 in s (seven conditions on seven
coefficients, ``fourth_derivative_weights``), error O(h^3), one order below
the scheme like the u_nn formula.
"""

from __future__ import annotations

from dataclasses import dataclass
from fractions import Fraction
from math import factorial
from typing import Dict, List

import numpy as np
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from .coupled import Grid, _classify, _face_of
from .stencils import laplacian, weighting


def fourth_derivative_weights():
    """(c_0..c_4, c_s, c_ss) of the one-sided u_ssss formula, as Fractions.

    Taylor: U_m = sum_k (m h)^k / k! u_k.  The combination
    sum c_m U_m + c_s h u_1 + c_ss h^2 u_2 must equal h^4 u_4 up to h^7:
    coefficients of u_3..u_6 involve c_1..c_4 only (a 4x4 system solved in
    exact arithmetic); those of u_0, u_1, u_2 then fix c_0, c_s and c_ss.
    """
    rows = [[Fraction(m ** k, factorial(k)) for m in range(1, 5)] for k in range(3, 7)]
    rhs = [Fraction(1) if k == 4 else Fraction(0) for k in range(3, 7)]
    # Gauss-Jordan elimination in Fractions
    A = [r[:] + [b] for r, b in zip(rows, rhs)]
    n = 4
    for c in range(n):
        piv = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        pv = A[c][c]
        A[c] = [v / pv for v in A[c]]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [a - f * b for a, b in zip(A[r], A[c])]
    c14 = [A[r][n] for r in range(n)]
    c0 = -sum(c14)
    cs = -sum(c * m for c, m in zip(c14, range(1, 5)))
    css = -sum(c * Fraction(m * m, 2) for c, m in zip(c14, range(1, 5)))
    return [c0] + c14, cs, css


@dataclass
class TriSystem:
    grid: Grid
    A: sps.csr_matrix
    F: np.ndarray
    n: int
    ng: int


@dataclass
class TriSolution:
    U: np.ndarray   # full grid, boundary = g_D
    V: np.ndarray   # full grid, boundary = Lap u data
    W: np.ndarray   # full grid, faces = Q, edges and corners = bilap
    Q: np.ndarray   # face layout (every face)


def assemble(data: Dict) -> TriSystem:
    """Assemble block rows (i)-(iv) for sampled data (``inputs.sample_triharmonic``)."""
    N = list(data["N"])
    grid = Grid(N, list(data["lo"]), list(data["hi"]))
    d = grid.dim
    h = grid.h
    n = grid.n_int
    ng = grid.n_gamma
    size = 3 * n + ng
    flat = lambda k: np.asarray(data[k], dtype=np.float64).reshape(-1)  # noqa: E731
    f, gD, vb, wb = flat("f"), flat("g_D"), flat("lap_gD"), flat("bilap")
    gN, gNN, lw = flat("g_N"), flat("g_NN"), flat("lapt_w")
    clamped = set(data.get("clamped") or ())

    L = laplacian(h)
    Mw = weighting(d)
    I = grid.interior_index_arrays()
    pid = grid.interior_flat(I)
    rows: List[np.ndarray] = []
    cols: List[np.ndarray] = []
    vals: List[np.ndarray] = []
    F = np.zeros(size)

    def add(r, c, v):
        rows.append(np.asarray(r, dtype=np.int64))
        cols.append(np.asarray(c, dtype=np.int64))
        vals.append(np.broadcast_to(np.asarray(v, dtype=np.float64), np.shape(r)).copy())

    ru, rv, rw = 3 * pid, 3 * pid + 1, 3 * pid + 2

    for off, c in L.items():
        j = [I[a] + off[a] for a in range(d)]
        inter, face, edge = _classify(grid, j)
        bnd = ~inter
        jf = grid.full_flat(j)
        ji = 3 * grid.interior_flat([jj[inter] for jj in j])
        # (i) L_h U, boundary U = g_D
        add(ru[inter], ji, c)
        np.add.at(F, ru[bnd], -c * gD[jf[bnd]])
        # (ii) L_h V, boundary V = Lap u
        add(rv[inter], ji + 1, c)
        np.add.at(F, rv[bnd], -c * vb[jf[bnd]])
        # (iii) L_h W, face W = Q, edge and corner W = Lap^2 u
        add(rw[inter], ji + 2, c)
        qf = _face_of(grid, j, face)
        add(rw[face], 3 * n + qf[face], c)
        np.add.at(F, rw[edge], -c * wb[jf[edge]])

    for off, c in Mw.items():
        j = [I[a] + off[a] for a in range(d)]
        inter, face, edge = _classify(grid, j)
        assert not np.any(edge)  # M reaches interior and face points only
        jf = grid.full_flat(j)
        ji = 3 * grid.interior_flat([jj[inter] for jj in j])
        # (i) - M V, face V data
        add(ru[inter], ji + 1, -c)
        np.add.at(F, ru[face], c * vb[jf[face]])
        # (ii) - M W, face W = Q
        add(rv[inter], ji + 2, -c)
        qf = _face_of(grid, j, face)
        add(rv[face], 3 * n + qf[face], -c)
        # (iii) right-hand side M f
        np.add.at(F, rw, c * f[jf])

    # (iv) augmented rows
    cw, cs, css = fourth_derivative_weights()
    for a in range(d):
        ha = h[a]
        wU = [float(cm) / ha ** 4 for cm in cw]
        ws, wss = float(cs) / ha ** 3, float(css) / ha ** 2
        for side in (0, 1):
            P = grid.face_point_indices(a, side)
            q = grid.face_flat(P, a, side)
            r = 3 * n + q
            pf = grid.full_flat(P)
            add(r, r, -1.0)
            if 2 * a + side not in clamped:
                F[r] = -wb[pf]
                continue
            step = 1 if side == 0 else -1
            for m in range(1, 5):
                jm = [P[b] if b != a else P[a] + step * m for b in range(d)]
                add(r, 3 * grid.interior_flat(jm), wU[m])
            # u_s along the inward normal is minus the outward g_N
            F[r] = -(wU[0] * gD[pf] + ws * (-gN[q]) + wss * gNN[q] + lw[q])

    A = sps.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(size, size))
    A.sum_duplicates()
    return TriSystem(grid, A, F, n, ng)


def solve_direct(sys_: TriSystem, data: Dict) -> TriSolution:
    """Solve the assembled system with SuperLU (FP64) and lay the result out on the full grid."""
    x = spla.splu(sys_.A.tocsc(), permc_spec="COLAMD").solve(sys_.F)
    g = sys_.grid
    n = sys_.n
    shape_int = tuple(m - 1 for m in reversed(g.N))
    shape_full = tuple(m + 1 for m in reversed(g.N))
    inner = tuple(slice(1, -1) for _ in range(g.dim))
    Q = x[3 * n:].copy()
    U = np.asarray(data["g_D"], dtype=float).reshape(shape_full).copy()
    V = np.asarray(data["lap_gD"], dtype=float).reshape(shape_full).copy()
    W = np.asarray(data["bilap"], dtype=float).reshape(shape_full).copy()
    U[inner] = x[0:3 * n:3].reshape(shape_int)
    V[inner] = x[1:3 * n:3].reshape(shape_int)
    W[inner] = x[2:3 * n:3].reshape(shape_int)
    Wf = W.reshape(-1)
    for a in range(g.dim):
        for side in (0, 1):
            P = g.face_point_indices(a, side)
            Wf[g.full_flat(P)] = Q[g.face_flat(P, a, side)]
    return TriSolution(U, V, W, Q)


class TriBlocks:
    """A11 = rows/columns of (U, V, W), A12, A21, A22 of the triharmonic system;
    the Schur complement S = A22 - A21 A11^-1 A12 and b = F2 - A21 A11^-1 F1."""

    def __init__(self, sys_: TriSystem):
        A = sys_.A.tocsr()
        m = 3 * sys_.n
        self.sys = sys_
        self.A11 = A[:m, :m].tocsc()
        self.A12 = A[:m, m:].tocsc()
        self.A21 = A[m:, :m].tocsr()
        self.A22 = A[m:, m:].tocsr()
        self.F1 = sys_.F[:m]
        self.F2 = sys_.F[m:]
        self.lu = spla.splu(self.A11, permc_spec="COLAMD")

    def schur_rhs(self):
        return self.F2 - self.A21 @ self.lu.solve(self.F1)

    def schur_dense(self):
        X = self.lu.solve(self.A12.toarray())
        return self.A22.toarray() - self.A21 @ X
