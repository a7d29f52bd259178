"""The coupled augmented HOC system, assembled and solved directly (oracle; test infrastructure).

Unknowns (Sec. 2.2, coupled block system): the interior values U and V of u
and v = alpha * Lap u, interleaved per interior point (U_p, V_p) to limit
fill, followed by the augmented boundary unknowns Q (the values of v on the
relative interiors of the clamped faces; fully clamped: every face).

Equations, one block row each:
  (i)   L_h U - M(V / alpha) = 0 at interior points            (Sec. 2.2, u-equation)
        boundary U = g_D moves to the right-hand side; V / alpha at a face
        point is Q / alpha there.  (Reading: the block zero in the first
        block row of the printed system hides only the Q columns that M does
        not reach; at the first interior layer M reaches the boundary value
        of v, which is Q.)
  (ii)  -L_h V + M(beta V / alpha) = M f at interior points     (Sec. 2.2, v-equation)
        V at face points is Q; V at edges and corners is the data v_edge
        (the Remark after the one-sided formula: there all of Lap u follows
        from g_D by tangential differentiation).
  (iii) on a clamped face (u_n = g_N, Eq. 2):
        alpha_p [ (delta_nn U)_p + lapt_gD_p ] - Q_p = 0 at face points p
        (Lemma 1's residual R_p), with the one-sided delta_nn of Sec. 2.2
        using U0 = g_D, U1..U3 interior and the outward g_N;
        on a Navier face (Lap u = g_L, Eq. 2): v = alpha g_L is data, the row
        is alpha_p g_L,p - Q_p = 0.

With this sign of block row (iii) the identity block is -I, so that the
algebraic residual R(Q) = A22 Q + A21 U(Q) - F2 of Lemma 1's proof equals the
printed R_p; then S_h = A22 - A21 A11^-1 A12 satisfies S_h Q = R(Q) - R(0) and
b = F2 - A21 A11^-1 F1 = -R(0) (Sec. 2.3, Eq. of the Schur system, Lemma 1).

Layouts follow ``paper_2609_16478_b300.inputs``: full-grid arrays in numpy
shape (N_z+1, N_y+1, N_x+1) (x fastest), face arrays in the order
x-, x+, y-, y+, z-, z+ with the lowest remaining axis fastest.
"""

from __future__ import annotations

import itertools
from dataclasses import dataclass
from typing import Dict, List, Optional, Sequence

import numpy as np
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from .stencils import laplacian, one_sided_weights, weighting


# ----------------------------------------------------------------------------
# grid bookkeeping
# ----------------------------------------------------------------------------

@dataclass
class Grid:
    N: List[int]
    lo: List[float]
    hi: List[float]

    @property
    def dim(self):
        return len(self.N)

    @property
    def h(self):
        return [(self.hi[a] - self.lo[a]) / self.N[a] for a in range(self.dim)]

    @property
    def n_int(self):
        return int(np.prod([n - 1 for n in self.N]))

    def face_sizes(self):
        out = []
        for a in range(self.dim):
            s = int(np.prod([self.N[b] - 1 for b in range(self.dim) if b != a]))
            out += [s, s]
        return out

    @property
    def n_gamma(self):
        return sum(self.face_sizes())

    def face_offsets(self):
        return np.concatenate([[0], np.cumsum(self.face_sizes())]).astype(np.int64)

    def interior_index_arrays(self):
        """Per-axis index arrays (values 1..N_a-1) of all interior points, x fastest."""
        rng = [np.arange(1, n) for n in self.N]
        g = np.meshgrid(*reversed(rng), indexing="ij")
        return [g[self.dim - 1 - a].reshape(-1) for a in range(self.dim)]

    def interior_flat(self, idx):
        """Linear interior index (x fastest) of interior points given per-axis indices."""
        out = np.zeros_like(idx[0])
        stride = 1
        for a in range(self.dim):
            out = out + (idx[a] - 1) * stride
            stride *= self.N[a] - 1
        return out

    def full_flat(self, idx):
        out = np.zeros_like(idx[0])
        stride = 1
        for a in range(self.dim):
            out = out + idx[a] * stride
            stride *= self.N[a] + 1
        return out

    def face_flat(self, idx, axis, side):
        """Index into the Q vector of face points (coordinate ``axis`` on the boundary)."""
        off = self.face_offsets()[2 * axis + side]
        out = np.zeros_like(idx[0])
        stride = 1
        for b in range(self.dim):
            if b == axis:
                continue
            out = out + (idx[b] - 1) * stride
            stride *= self.N[b] - 1
        return off + out

    def face_point_indices(self, axis, side):
        """Per-axis index arrays of a face's relative-interior points, in Q order."""
        rest = [b for b in range(self.dim) if b != axis]
        rng = [np.arange(1, self.N[b]) for b in rest]
        g = np.meshgrid(*reversed(rng), indexing="ij")
        g = list(reversed(g))
        out = [None] * self.dim
        for i, b in enumerate(rest):
            out[b] = g[i].reshape(-1)
        n = out[rest[0]].size
        out[axis] = np.full(n, 0 if side == 0 else self.N[axis], dtype=np.int64)
        return out


def _classify(grid: Grid, j):
    """Split neighbour points into interior / face-interior / edge-or-corner masks."""
    nb = np.zeros_like(j[0])
    for a in range(grid.dim):
        nb = nb + ((j[a] == 0) | (j[a] == grid.N[a])).astype(np.int64)
    return nb == 0, nb == 1, nb >= 2


def _face_of(grid: Grid, j, mask):
    """For face points (mask), their Q index."""
    q = np.full(j[0].shape, -1, dtype=np.int64)
    for a in range(grid.dim):
        for side, val in ((0, 0), (1, grid.N[a])):
            m = mask & (j[a] == val)
            if np.any(m):
                q[m] = grid.face_flat([jj[m] for jj in j], a, side)
    return q


# ----------------------------------------------------------------------------
# assembly
# ----------------------------------------------------------------------------

@dataclass
class Coupled:
    grid: Grid
    A: sps.csr_matrix           # full coupled matrix, size 2n + n_gamma
    F: np.ndarray               # right-hand side
    n: int                      # interior points
    ng: int                     # augmented unknowns

    @property
    def iu(self):
        return np.arange(self.n) * 2

    @property
    def iv(self):
        return np.arange(self.n) * 2 + 1


def assemble(data: Dict, N=None, lo=None, hi=None) -> Coupled:
    """Assemble the coupled system for sampled data (see ``inputs.sample``).

    data holds full-grid arrays alpha, f, g_D, v_edge and face arrays g_N and
    lapt_gD (any of the data arrays may be None, meaning zero); optionally
    beta (a number or a full-grid array; default 0), navier (the face ids
    2 * axis + side of the Navier faces; default none) and the face array
    g_L (Lap u on the faces; read on Navier faces).
    """
    N = list(N if N is not None else data["N"])
    lo = list(lo if lo is not None else data["lo"])
    hi = list(hi if hi is not None else data["hi"])
    grid = Grid(N, lo, hi)
    d = grid.dim
    h = grid.h
    n = grid.n_int
    ng = grid.n_gamma
    size = 2 * n + ng

    def flat(key):
        a = data.get(key)
        if a is None:
            return None
        return np.asarray(a, dtype=np.float64).reshape(-1)

    alpha = flat("alpha")
    f = flat("f")
    gD = flat("g_D")
    vE = flat("v_edge")
    gN = flat("g_N")
    lapt = flat("lapt_gD")
    zero_full = np.zeros(int(np.prod([m + 1 for m in N])))
    f = zero_full if f is None else f
    gD = zero_full if gD is None else gD
    vE = zero_full if vE is None else vE
    gN = np.zeros(ng) if gN is None else gN
    lapt = np.zeros(ng) if lapt is None else lapt
    beta = data.get("beta", 0.0)
    beta = np.broadcast_to(np.asarray(beta if beta is not None else 0.0, dtype=np.float64).reshape(-1)
                           if np.ndim(beta) else np.float64(beta), zero_full.shape)
    navier = set(data.get("navier") or ())
    gL = flat("g_L")
    gL = np.zeros(ng) if gL is None else gL

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

    ru = 2 * pid        # u-equation rows
    rv = 2 * pid + 1    # v-equation rows

    for off, c in L.items():
        j = [I[a] + off[a] for a in range(d)]
        inter, face, edge = _classify(grid, j)
        jf = grid.full_flat(j)
        # (i) L_h U: interior U unknowns, boundary U = g_D to the right-hand side
        add(ru[inter], 2 * grid.interior_flat([jj[inter] for jj in j]), c)
        bnd = ~inter
        np.add.at(F, ru[bnd], -c * gD[jf[bnd]])
        # (ii) -L_h V: interior V unknowns, face V = Q unknowns, edge/corner V = data
        add(rv[inter], 2 * grid.interior_flat([jj[inter] for jj in j]) + 1, -c)
        qf = _face_of(grid, j, face)
        add(rv[face], 2 * n + qf[face], -c)
        np.add.at(F, rv[edge], c * vE[jf[edge]])

    for off, c in Mw.items():
        j = [I[a] + off[a] for a in range(d)]
        inter, face, edge = _classify(grid, j)
        assert not np.any(edge)  # M only reaches interior and face points
        jf = grid.full_flat(j)
        # (i) - M(V / alpha)
        add(ru[inter], 2 * grid.interior_flat([jj[inter] for jj in j]) + 1, -c / alpha[jf[inter]])
        qf = _face_of(grid, j, face)
        add(ru[face], 2 * n + qf[face], -c / alpha[jf[face]])
        # (ii) + M(beta V / alpha)
        ba = beta[jf] / alpha[jf]
        add(rv[inter], 2 * grid.interior_flat([jj[inter] for jj in j]) + 1, c * ba[inter])
        add(rv[face], 2 * n + qf[face], c * ba[face])
        # (ii) right-hand side M f (f sampled on the full grid, boundary included)
        np.add.at(F, rv, c * f[jf])

    # (iii) augmented equations
    for a in range(d):
        (w0, w1, w2, w3), wg = one_sided_weights(h[a])
        for side in (0, 1):
            P = grid.face_point_indices(a, side)
            q = grid.face_flat(P, a, side)
            r = 2 * n + q
            pf = grid.full_flat(P)
            al = alpha[pf]
            if 2 * a + side in navier:
                add(r, r, -1.0)
                F[r] = -al * gL[q]
                continue
            step = 1 if side == 0 else -1
            for m, w in ((1, w1), (2, w2), (3, w3)):
                jm = [P[b] if b != a else P[a] + step * m for b in range(d)]
                add(r, 2 * grid.interior_flat(jm), al * w)
            add(r, r, -1.0)
            F[r] = -al * (w0 * gD[pf] + wg * gN[q] + lapt[q])

    A = sps.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(size, size))
    A.sum_duplicates()
    return Coupled(grid, A, F, n, ng)


# ----------------------------------------------------------------------------
# direct solve and post-processing
# ----------------------------------------------------------------------------

@dataclass
class Solution:
    U: np.ndarray       # full grid, boundary = g_D
    V: np.ndarray       # full grid, faces = Q, edges/corners = v_edge
    Q: np.ndarray       # face values
    U_int: np.ndarray   # interior (x fastest), numpy shape reversed
    V_int: np.ndarray


def solve_direct(sys_: Coupled, data: Dict) -> Solution:
    """Solve the assembled coupled system with SuperLU (FP64)."""
    A = sys_.A.tocsc()
    lu = spla.splu(A, permc_spec="COLAMD")
    x = lu.solve(sys_.F)
    return unpack(sys_, data, x)


def unpack(sys_: Coupled, data: Dict, x: np.ndarray) -> Solution:
    g = sys_.grid
    n = sys_.n
    shape_int = tuple(m - 1 for m in reversed(g.N))
    shape_full = tuple(m + 1 for m in reversed(g.N))
    U_int = x[0:2 * n:2].reshape(shape_int)
    V_int = x[1:2 * n:2].reshape(shape_int)
    Q = x[2 * n:].copy()
    gD = np.asarray(data["g_D"], dtype=float).reshape(shape_full) if data.get("g_D") is not None else np.zeros(shape_full)
    vE = np.asarray(data["v_edge"], dtype=float).reshape(shape_full) if data.get("v_edge") is not None else np.zeros(shape_full)
    U = gD.copy()
    inner = tuple(slice(1, -1) for _ in range(g.dim))
    U[inner] = U_int
    V = vE.copy()
    V[inner] = V_int
    Vf = V.reshape(-1)
    for a in range(g.dim):
        for side in (0, 1):
            P = g.face_point_indices(a, side)
            q = g.face_flat(P, a, side)
            Vf[g.full_flat(P)] = Q[q]
    return Solution(U, V, Q, U_int, V_int)


# ----------------------------------------------------------------------------
# Schur complement from the assembled blocks (Sec. 2.3)
# ----------------------------------------------------------------------------

class Blocks:
    """The partition A11, A12, A21, A22 of the coupled system with A11 factored."""

    def __init__(self, sys_: Coupled):
        A = sys_.A.tocsr()
        m = 2 * sys_.n
        self.sys = sys_
        self.A11 = A[:m, :m].tocsc()
        self.A12 = A[:m, m:].tocsc()
        self.A21 = A[m:, :m].tocsr()
        self.A22 = A[m:, m:].tocsr()
        self.F1 = sys_.F[:m]
        self.F2 = sys_.F[m:]
        self.lu = spla.splu(self.A11, permc_spec="COLAMD")

    def U_of(self, Q):
        """The (U, V) solution of block row 1 for given Q: A11 X = F1 - A12 Q."""
        return self.lu.solve(self.F1 - self.A12 @ Q)

    def residual(self, Q):
        """Lemma 1's algebraic residual R(Q) = A22 Q + A21 X(Q) - F2."""
        return self.A22 @ Q + self.A21 @ self.U_of(Q) - self.F2

    def schur_apply(self, Q):
        """S_h Q = A22 Q - A21 A11^-1 A12 Q (no data terms)."""
        return self.A22 @ Q - self.A21 @ self.lu.solve(self.A12 @ Q)

    def schur_rhs(self):
        """b = F2 - A21 A11^-1 F1."""
        return self.F2 - self.A21 @ self.lu.solve(self.F1)

    def schur_dense(self):
        """The explicit Schur complement (small grids only)."""
        ng = self.sys.ng
        S = np.empty((ng, ng))
        A12 = self.A12.toarray()
        X = self.lu.solve(A12)
        S[:] = self.A22.toarray() - self.A21 @ X
        return S


def solve_schur_dense(sys_: Coupled, data: Dict) -> Solution:
    """Solve via the explicit Schur complement (Sec. 2.3), then recover U and V."""
    B = Blocks(sys_)
    S = B.schur_dense()
    Q = np.linalg.solve(S, B.schur_rhs())
    X = B.U_of(Q)
    return unpack(sys_, data, np.concatenate([X, Q]))


# ----------------------------------------------------------------------------
# single-operator helpers used by component tests
# ----------------------------------------------------------------------------

def laplacian_matrix(N: Sequence[int], lo=None, hi=None) -> sps.csr_matrix:
    """L_h on interior points with zero Dirichlet values (x fastest)."""
    d = len(N)
    lo = list(lo) if lo is not None else [0.0] * d
    hi = list(hi) if hi is not None else [1.0] * d
    g = Grid(list(N), lo, hi)
    I = g.interior_index_arrays()
    pid = g.interior_flat(I)
    rows, cols, vals = [], [], []
    for off, c in laplacian(g.h).items():
        j = [I[a] + off[a] for a in range(d)]
        inter, _, _ = _classify(g, j)
        rows.append(pid[inter])
        cols.append(g.interior_flat([jj[inter] for jj in j]))
        vals.append(np.full(int(inter.sum()), c))
    n = g.n_int
    return sps.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def poisson_solve(N: Sequence[int], rhs_int: np.ndarray, lo=None, hi=None) -> np.ndarray:
    """Solve L_h W = rhs on interior points with W = 0 on the boundary (SuperLU)."""
    A = laplacian_matrix(N, lo, hi).tocsc()
    w = spla.spsolve(A, np.asarray(rhs_int, dtype=float).reshape(-1))
    return w.reshape(np.shape(rhs_int))
