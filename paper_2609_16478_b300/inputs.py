"""Seeded synthetic problem generators (inputs only: nothing of the method).

Every workload of the augmented HOC method is a clamped problem
    -Laplace(alpha * Laplace u) = f   in a box                    (Sec. 2, Eq. 1, beta = 0)
    u = g_D on the whole boundary, u_n = g_N on every face        (Eq. 2, fully clamped)
whose data are manufactured analytically from an exact u and a coefficient
alpha.  This module turns such a definition into sampled arrays in the layout
the C ABI uses; both the CUDA path and the CPU oracle consume them.  It holds
no discrete operator, no solver step and nothing else of the method.

Layouts (shared convention of the library's boundary):
  * full-grid arrays have (N_a + 1) points per axis a, x fastest; numpy shape
    is therefore reversed: (N_z+1, N_y+1, N_x+1) in 3D, (N_y+1, N_x+1) in 2D;
  * face arrays (g_N, lapt_gD, Q) list the relative-interior points of the
    faces in the order x-, x+, y-, y+, z-, z+; within a face the remaining
    axes keep the same order (lowest axis fastest).

The random coefficient fields follow a fixed recipe: phi(x) is a sum of M
cosines cos(2 pi k_m . x + theta_m) with integer wave vectors 0 <= k_m,a <= K
(k_m != 0), amplitudes c_m ~ U(-1, 1) and phases theta_m ~ U(0, 2 pi) drawn
from numpy's default_rng(seed); phi is normalised by its maximum modulus on a
fixed lattice (1025 points per axis in 2D, 129 in 3D) so that the coefficient
does not depend on the solve resolution, and alpha = 1 + A * phi / max|phi|.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np
import sympy as sp

X = sp.symbols("x y z", real=True)

__all__ = [
    "Problem", "fourier_alpha", "config_problem", "sample", "face_sizes",
    "n_gamma", "WORKLOADS", "TriProblem", "triharmonic_problem", "sample_triharmonic",
]


# ----------------------------------------------------------------------------
# coefficient fields
# ----------------------------------------------------------------------------

def fourier_modes(dim: int, M: int, K: int, seed: int):
    """Draw the M Fourier modes of a seeded smooth random field."""
    rng = np.random.default_rng(seed)
    modes = []
    for _ in range(M):
        while True:
            k = rng.integers(0, K + 1, size=dim)
            if np.any(k != 0):
                break
        c = rng.uniform(-1.0, 1.0)
        th = rng.uniform(0.0, 2.0 * math.pi)
        modes.append((tuple(int(v) for v in k), float(c), float(th)))
    return modes


def fourier_alpha(dim: int, M: int, K: int, A: float, seed: int) -> sp.Expr:
    """alpha = 1 + A * phi / max|phi| with phi a seeded sum of M cosines."""
    modes = fourier_modes(dim, M, K, seed)
    xs = X[:dim]
    phi = sum(sp.Float(c) * sp.cos(2 * sp.pi * sum(int(k[a]) * xs[a] for a in range(dim)) + sp.Float(th))
              for k, c, th in modes)
    L = 1024 if dim == 2 else 128
    t = np.linspace(0.0, 1.0, L + 1)
    grids = np.meshgrid(*([t] * dim), indexing="ij")
    val = np.zeros_like(grids[0])
    for k, c, th in modes:
        val += c * np.cos(2 * np.pi * sum(k[a] * grids[a] for a in range(dim)) + th)
    mx = float(np.max(np.abs(val)))
    return 1 + sp.Float(A) * phi / sp.Float(mx)


# ----------------------------------------------------------------------------
# problem definitions
# ----------------------------------------------------------------------------

@dataclass
class Problem:
    """A clamped problem: exact u (optional), alpha, and data overrides.

    f defaults to -Laplace(alpha * Laplace u) applied analytically; g_D, g_N,
    the tangential Laplacian of g_D on faces and alpha*Laplace(u) on edges and
    corners default to the exact u's traces.  Problems without an exact
    solution (the cavity, the plate) give their data explicitly.
    """

    name: str
    dim: int
    alpha: sp.Expr
    u: Optional[sp.Expr] = None
    f_grid: Optional[Callable] = None          # f_grid(N, lo, hi) -> full-grid array
    gN_face: Optional[Callable] = None         # gN_face(axis, side, coords) -> values
    lo: Tuple[float, ...] = (0.0, 0.0, 0.0)
    hi: Tuple[float, ...] = (1.0, 1.0, 1.0)
    note: str = ""
    beta: object = 0.0                         # beta of Eq. 1: a number or a sympy expression
    navier: Tuple[int, ...] = ()               # Navier faces (2 * axis + side): Lap u = g_L there

    def exprs(self) -> Dict[str, sp.Expr]:
        xs = X[: self.dim]
        out = {"alpha": self.alpha}
        if self.u is not None:
            u = self.u
            lap = sum(sp.diff(u, v, 2) for v in xs)
            w = self.alpha * lap
            out["u"] = u
            out["lap"] = lap
            out["v"] = w
            out["f"] = -sum(sp.diff(w, v, 2) for v in xs) + sp.sympify(self.beta) * lap
            out["beta"] = sp.sympify(self.beta)
            for a, v in enumerate(xs):
                out[f"du{a}"] = sp.diff(u, v)
                out[f"d2u{a}"] = sp.diff(u, v, 2)
        return out


def _sinsq(v):
    return sp.sin(sp.pi * v) ** 2


def config_problem(name: str) -> Problem:
    """The named synthetic workloads."""
    x, y, z = X
    if name == "smooth2d":
        # 2D, unit square, alpha = 1 + 0.5 sin(2 pi x) sin(2 pi y), u = sin^2 sin^2
        return Problem(name, 2, 1 + sp.Rational(1, 2) * sp.sin(2 * sp.pi * x) * sp.sin(2 * sp.pi * y),
                       _sinsq(x) * _sinsq(y))
    if name == "fourier2d":
        # 2D, alpha = 1 + 0.4 * (8 seeded modes, |k| <= 6), u = sin^2 sin^2 cos(pi x)
        return Problem(name, 2, fourier_alpha(2, 8, 6, 0.4, 1), _sinsq(x) * _sinsq(y) * sp.cos(sp.pi * x))
    if name == "fourier3d":
        return Problem(name, 3, fourier_alpha(3, 6, 4, 0.4, 2), _sinsq(x) * _sinsq(y) * _sinsq(z))
    if name == "fourier3d_k32":
        k = 32
        u = _sinsq(x) * _sinsq(y) * _sinsq(z) * sp.sin(k * sp.pi * x) * sp.sin(k * sp.pi * y) * sp.sin(k * sp.pi * z)
        return Problem(name, 3, fourier_alpha(3, 6, 4, 0.5, 3), u)
    if name == "sincos2d":
        # nonzero g_D, g_N, tangential Laplacian and corner v: exercises every data term
        return Problem(name, 2, 1 + x ** 2 + y ** 2, sp.sin(3 * x) * sp.cos(y + sp.Rational(1, 3)))
    if name == "sincos3d":
        return Problem(name, 3, 1 + x ** 2 + y ** 2 + z ** 2,
                       sp.sin(3 * x) * sp.cos(y + sp.Rational(1, 3)) * sp.sin(2 * z + sp.Rational(1, 2)))
    if name == "poly2d":
        # degree-4 polynomial with nonzero data everywhere and constant alpha
        return Problem(name, 2, sp.Integer(1), x ** 4 + x * y ** 3 - 2 * x ** 2 * y + y + 1)
    if name.startswith("singular2d"):
        # Example 1 (Sec. 4.1, Table 1): -eps Lap^2 u + Lap u = f on the unit
        # square, alpha = eps, beta = 1, clamped on x = 0 and Navier on the
        # other faces; name "singular2d" (eps = 1e-4) or "singular2d_eps1e-5"
        eps = sp.Float(name.split("_eps")[1]) if "_eps" in name else sp.Float("1e-4")
        u = 256 * (x ** 2 + eps * (1 - sp.exp(-x / sp.sqrt(eps))) ** 2) * (x - 1) ** 2 * y ** 2 * (y - 1) ** 2
        return Problem(name, 2, eps, u, beta=1.0, navier=(1, 2, 3))
    if name.startswith("peak3d") or name.startswith("sincos3d_var"):
        # Examples 2 and 3 (Sec. 4.1, Tables 2-3): alpha = x^2 + y^2 + z^2 + 1,
        # beta = x + y + z + 10, clamped on x = 0 and Navier on the other faces;
        # "peak3d_q10_p0.2", "peak3d_q5_p1", "sincos3d_var_5_1_5", "sincos3d_var_25_5_25"
        alpha = x ** 2 + y ** 2 + z ** 2 + 1
        beta = x + y + z + 10
        par = name.split("_")
        if name.startswith("peak3d"):
            q, p = sp.Rational(par[1][1:]), sp.Rational(par[2][1:])
            u = (x ** 2 - x) * (y ** 2 - y) * (z ** 2 - z) * sp.exp(q * ((x - sp.Rational(1, 2)) ** 2 +
                                                                         (y - sp.Rational(1, 2)) ** 2 + (z - p) ** 2))
        else:
            k1, k2, k3 = (int(v) for v in par[2:5])
            u = sp.sin(k1 * x) * sp.cos(k2 * y) * sp.sin(k3 * z)
        return Problem(name, 3, alpha, u, beta=beta, navier=(1, 2, 3, 4, 5))
    if name.startswith("classic3d"):
        # Table 4's timing problems: the classical biharmonic (alpha = 1, beta = 0)
        # with Example 2's (q, p) = (5, 1) or Example 3's (25, 5, 25) solution;
        # "classic3d_peak" or "classic3d_sincos"; clamped on x = 0, Navier elsewhere
        if name.endswith("peak"):
            u = (x ** 2 - x) * (y ** 2 - y) * (z ** 2 - z) * sp.exp(5 * ((x - sp.Rational(1, 2)) ** 2 +
                                                                         (y - sp.Rational(1, 2)) ** 2 + (z - 1) ** 2))
        else:
            u = sp.sin(25 * x) * sp.cos(5 * y) * sp.sin(25 * z)
        return Problem(name, 3, sp.Integer(1), u, navier=(1, 2, 3, 4, 5))
    if name == "varbeta2d":
        # variable alpha and beta (beta/alpha not constant), one Navier face
        return Problem(name, 2, 1 + x ** 2 + y ** 2, sp.sin(3 * x) * sp.cos(y + sp.Rational(1, 3)),
                       beta=5 + x + 2 * y, navier=(1,))
    if name == "navier2d":
        # variable coefficient, beta = 0, clamped on x- and y-, Navier on x+ and y+
        return Problem(name, 2, 1 + x ** 2 + y ** 2, sp.sin(3 * x) * sp.cos(y + sp.Rational(1, 3)), navier=(1, 3))
    if name == "navier3d":
        return Problem(name, 3, 1 + x ** 2 + y ** 2 + z ** 2,
                       sp.sin(3 * x) * sp.cos(y + sp.Rational(1, 3)) * sp.sin(2 * z + sp.Rational(1, 2)),
                       beta=0.0, navier=(0, 3, 5))
    if name == "shift2d":
        # constant alpha and beta (the shifted-eigenvalue case) with nonzero data on every face
        return Problem(name, 2, sp.Float(2.0), sp.sin(3 * x) * sp.cos(y + sp.Rational(1, 3)), beta=50.0,
                       navier=(2,))
    if name == "cavity":
        # lid-driven cavity streamfunction: f = 0, u = 0, u_y = 1 on y = 1 (Sec. 4, Table 6)
        def gN(axis, side, coords):
            return np.ones_like(coords[0]) if (axis == 1 and side == 1) else np.zeros_like(coords[0])
        return Problem(name, 2, sp.Integer(1), None, f_grid=_zero_f, gN_face=gN)
    if name == "plate":
        # clamped plate under a unit central load; the library solves -Lap^2 u = f, so f = -load.
        return Problem(name, 2, sp.Integer(1), None, f_grid=_plate_f, gN_face=_zero_gN,
                       note="trapezoid-weighted 3x3 load of total mass 1")
    raise KeyError(name)


def _zero_f(N, lo, hi):
    return np.zeros(tuple(n + 1 for n in reversed(N)))


def _zero_gN(axis, side, coords):
    return np.zeros_like(coords[0])


def _plate_f(N, lo, hi):
    """-(unit load) spread over the 3x3 grid points around the centre.

    The load density is 1/(4h^2) on |x-1/2| <= h, |y-1/2| <= h; the nine grid
    points of that closed square get trapezoid weights (1, 1/2, 1/4) so that
    the discrete load h^2 * sum f is exactly 1.
    """
    Nx, Ny = N
    assert Nx % 2 == 0 and Ny % 2 == 0
    hx = (hi[0] - lo[0]) / Nx
    hy = (hi[1] - lo[1]) / Ny
    f = np.zeros((Ny + 1, Nx + 1))
    cx, cy = Nx // 2, Ny // 2
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            w = (0.5 if di else 1.0) * (0.5 if dj else 1.0)
            f[cy + dj, cx + di] = -w / (4.0 * hx * hy)
    return f


WORKLOADS = {
    "smooth2d": dict(dim=2, Ns=[64]),
    "fourier2d": dict(dim=2, Ns=[256, 512, 1024, 2048, 4096]),
    "fourier3d": dict(dim=3, Ns=[256, 512]),
    "fourier3d_k32": dict(dim=3, Ns=[1024]),
}


# ----------------------------------------------------------------------------
# sampling
# ----------------------------------------------------------------------------

def face_sizes(N: Sequence[int]) -> List[int]:
    """Number of relative-interior points of each face, in face order."""
    d = len(N)
    out = []
    for a in range(d):
        s = 1
        for b in range(d):
            if b != a:
                s *= N[b] - 1
        out += [s, s]
    return out


def n_gamma(N: Sequence[int]) -> int:
    return sum(face_sizes(N))


_TORCH_MAP = None


def _lamb(expr, dim, backend):
    xs = X[:dim]
    if backend == "numpy":
        return sp.lambdify(xs, expr, modules="numpy", cse=True)
    import torch
    global _TORCH_MAP
    if _TORCH_MAP is None:
        _TORCH_MAP = {"sin": torch.sin, "cos": torch.cos, "exp": torch.exp, "sqrt": torch.sqrt,
                      "pi": math.pi, "E": math.e}
    return sp.lambdify(xs, expr, modules=[_TORCH_MAP], cse=True)


def _coords(N, lo, hi, dim):
    return [lo[a] + (hi[a] - lo[a]) * np.arange(N[a] + 1) / N[a] for a in range(dim)]


def _eval_full(fn, N, lo, hi, dim, backend, device, chunk_pts=1 << 24):
    """Evaluate fn on the full (N+1)^d grid, chunked over the slowest axis."""
    c = _coords(N, lo, hi, dim)
    shape = tuple(N[a] + 1 for a in reversed(range(dim)))
    if backend == "numpy":
        out = np.empty(shape)
        plane = int(np.prod(shape[1:]))
        step = max(1, chunk_pts // plane)
        for s in range(0, shape[0], step):
            e = min(shape[0], s + step)
            sl = [c[a] for a in range(dim)]
            sl[dim - 1] = c[dim - 1][s:e]
            g = np.meshgrid(*reversed(sl), indexing="ij")  # slowest first
            args = list(reversed(g))
            out[s:e] = np.broadcast_to(fn(*args), g[0].shape)
        return out
    import torch
    out = torch.empty(shape, dtype=torch.float64, device=device)
    tc = [torch.tensor(v, dtype=torch.float64, device=device) for v in c]
    plane = int(np.prod(shape[1:]))
    step = max(1, chunk_pts // plane)
    for s in range(0, shape[0], step):
        e = min(shape[0], s + step)
        sl = list(tc)
        sl[dim - 1] = tc[dim - 1][s:e]
        g = torch.meshgrid(*reversed(sl), indexing="ij")
        args = list(reversed(g))
        val = fn(*args)
        if not torch.is_tensor(val):
            val = torch.full(g[0].shape, float(val), dtype=torch.float64, device=device)
        out[s:e] = val
    return out


def face_coords(N, lo, hi, axis, side):
    """Coordinates (one array per axis) of a face's relative-interior points."""
    dim = len(N)
    c = _coords(N, lo, hi, dim)
    rest = [b for b in range(dim) if b != axis]
    g = np.meshgrid(*[c[b][1:-1] for b in reversed(rest)], indexing="ij")
    g = list(reversed(g))  # g[i] varies along rest[i]; rest[0] fastest
    out = [None] * dim
    for i, b in enumerate(rest):
        out[b] = g[i].reshape(-1)
    n = out[rest[0]].size
    out[axis] = np.full(n, c[axis][0] if side == 0 else c[axis][-1])
    return out


def _edge_mask(N, dim):
    shape = tuple(N[a] + 1 for a in reversed(range(dim)))
    cnt = np.zeros(shape, dtype=np.int8)
    for a in range(dim):
        idx = [slice(None)] * dim
        ax = dim - 1 - a
        idx[ax] = 0
        cnt[tuple(idx)] += 1
        idx[ax] = N[a]
        cnt[tuple(idx)] += 1
    return cnt


def sample(prob: Problem, N: Sequence[int], lo=None, hi=None, backend: str = "numpy",
           device=None, with_exact: bool = True) -> Dict[str, object]:
    """Sample a problem on a grid with N[a] intervals per axis.

    Returns full-grid arrays alpha, f, g_D (boundary values of u; interior
    entries 0), v_edge (alpha * Laplace u at edge and corner points; 0
    elsewhere), face arrays g_N (outward normal derivative) and lapt_gD (sum of
    the tangential second derivatives of g_D), and, when the problem has one,
    the exact u and v = alpha * Laplace u on the full grid.  ``backend`` is
    "numpy" (host float64) or "torch" (float64 tensors on ``device``); face
    arrays are always computed on the host and converted.
    """
    dim = prob.dim
    N = [int(n) for n in N]
    lo = tuple(lo) if lo is not None else prob.lo[:dim]
    hi = tuple(hi) if hi is not None else prob.hi[:dim]
    ex = prob.exprs()
    out: Dict[str, object] = {"dim": dim, "N": N, "lo": lo, "hi": hi, "name": prob.name}

    def full(key):
        return _eval_full(_lamb(ex[key], dim, backend), N, lo, hi, dim, backend, device)

    out["alpha"] = full("alpha")
    if prob.f_grid is not None:
        f = prob.f_grid(N, lo, hi)
        out["f"] = f if backend == "numpy" else _to_t(f, device)
    else:
        out["f"] = full("f")

    # boundary data from exact u (host side; boundary-only sizes)
    fs = []
    gN = []
    lapt = []
    gL = []
    for a in range(dim):
        for side in (0, 1):
            pc = face_coords(N, lo, hi, a, side)
            fs.append(pc[0].size)
            if prob.u is not None:
                du = _lamb(ex[f"du{a}"], dim, "numpy")(*pc)
                val = np.broadcast_to(np.asarray(du, dtype=float), pc[0].shape).copy()
                gN.append(-val if side == 0 else val)
                lt = np.zeros(pc[0].size)
                for b in range(dim):
                    if b != a:
                        lt += np.broadcast_to(np.asarray(_lamb(ex[f"d2u{b}"], dim, "numpy")(*pc), float), lt.shape)
                lapt.append(lt)
                gL.append(np.broadcast_to(np.asarray(_lamb(ex["lap"], dim, "numpy")(*pc), float), lt.shape).copy())
            else:
                gN.append(np.asarray(prob.gN_face(a, side, pc), dtype=float))
                lapt.append(np.zeros(pc[0].size))
                gL.append(np.zeros(pc[0].size))
    gN = np.concatenate(gN)
    lapt = np.concatenate(lapt)
    gL = np.concatenate(gL)

    cnt = _edge_mask(N, dim)
    if prob.u is not None:
        u_full = full("u")
        v_full = full("v")
        if backend == "numpy":
            bmask = cnt > 0
            gD = np.where(bmask, u_full, 0.0)
            vE = np.where(cnt >= 2, v_full, 0.0)
        else:
            import torch
            cm = torch.from_numpy(cnt).to(device)
            gD = torch.where(cm > 0, u_full, torch.zeros_like(u_full))
            vE = torch.where(cm >= 2, v_full, torch.zeros_like(v_full))
        if with_exact:
            out["u_exact"] = u_full
            out["v_exact"] = v_full
        else:
            del u_full, v_full
    else:
        z = np.zeros(tuple(n + 1 for n in reversed(N)))
        gD = z if backend == "numpy" else _to_t(z, device)
        vE = z.copy() if backend == "numpy" else _to_t(z, device)
    out["g_D"] = gD
    out["v_edge"] = vE
    out["g_N"] = gN if backend == "numpy" else _to_t(gN, device)
    out["lapt_gD"] = lapt if backend == "numpy" else _to_t(lapt, device)
    if isinstance(prob.beta, sp.Expr) and not prob.beta.is_number:
        out["beta"] = full("beta")
    else:
        out["beta"] = float(prob.beta)
    out["navier"] = tuple(prob.navier)
    if prob.navier:
        out["g_L"] = gL if backend == "numpy" else _to_t(gL, device)
    return out


def _to_t(a, device):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=device)


# ----------------------------------------------------------------------------
# triharmonic problems: Lap^3 u = f (the paper's triharmonic extension, Table 5)
# ----------------------------------------------------------------------------

@dataclass
class TriProblem:
    """Lap^3 u = f in a box with u, u_n and u_nn given on the clamped faces and
    u, Lap u and Lap^2 u given on the other (simply supported) faces; all data
    are traces of the exact u."""

    name: str
    dim: int
    u: sp.Expr
    clamped: Tuple[int, ...] = (0,)            # face ids 2 * axis + side
    lo: Tuple[float, ...] = (0.0, 0.0, 0.0)
    hi: Tuple[float, ...] = (1.0, 1.0, 1.0)


def triharmonic_problem(name: str) -> TriProblem:
    """"tri3d_5_1_5", "tri3d_25_5_25": u = sin(k1 x) cos(k2 y) sin(k3 z),
    clamped on x = 0 (the setting of Table 5); "tripoly3d", "tripoly2d":
    polynomials of degree 5 with nonzero data of every kind, clamped on two
    faces; "trisin2d": a smooth 2D solution clamped on x = 0."""
    x, y, z = X
    if name.startswith("tri3d_"):
        k1, k2, k3 = (int(v) for v in name.split("_")[1:4])
        return TriProblem(name, 3, sp.sin(k1 * x) * sp.cos(k2 * y) * sp.sin(k3 * z), clamped=(0,))
    if name == "tripoly3d":
        u = x ** 5 - 2 * x ** 3 * y ** 2 + x * y * z ** 3 + y ** 4 * z - z ** 5 / 3 + x ** 2 * z + y - 1
        return TriProblem(name, 3, u, clamped=(0, 3))
    if name == "tripoly2d":
        u = x ** 5 - 3 * x ** 3 * y ** 2 + 2 * x * y ** 4 + y ** 5 / 5 + x ** 2 * y - x + 2
        return TriProblem(name, 2, u, clamped=(0, 2))
    if name == "trisin2d":
        return TriProblem(name, 2, sp.sin(3 * x + sp.Rational(1, 4)) * sp.cos(2 * y), clamped=(0,))
    raise KeyError(name)


def sample_triharmonic(prob: TriProblem, N: Sequence[int], lo=None, hi=None, backend: str = "numpy",
                       device=None) -> Dict[str, object]:
    """Sample a triharmonic problem: full-grid arrays f (= Lap^3 u), u_exact, and
    the boundary data g_D (u), lap_gD (Lap u) and bilap (Lap^2 u), each with
    its interior entries 0; face arrays g_N (outward normal derivative), g_NN
    (second normal derivative) and lapt_w (2 Lap_t u_nn + Lap_t^2 u, Lap_t the
    sum of the tangential second derivatives), in the layouts of ``sample``."""
    dim = prob.dim
    N = [int(n) for n in N]
    lo = tuple(lo) if lo is not None else prob.lo[:dim]
    hi = tuple(hi) if hi is not None else prob.hi[:dim]
    xs = X[:dim]
    u = prob.u
    lap = lambda e: sum(sp.diff(e, v, 2) for v in xs)  # noqa: E731
    lu = lap(u)
    l2u = lap(lu)
    out: Dict[str, object] = {"dim": dim, "N": N, "lo": lo, "hi": hi, "name": prob.name,
                              "clamped": tuple(prob.clamped), "triharmonic": True}

    def full(expr):
        return _eval_full(_lamb(expr, dim, backend), N, lo, hi, dim, backend, device)

    out["f"] = full(lap(l2u))
    u_full = full(u)
    cnt = _edge_mask(N, dim)
    if backend == "numpy":
        bm = cnt > 0
        out["g_D"] = np.where(bm, u_full, 0.0)
        out["lap_gD"] = np.where(bm, full(lu), 0.0)
        out["bilap"] = np.where(bm, full(l2u), 0.0)
    else:
        import torch
        bm = torch.from_numpy(cnt).to(device) > 0
        zero = torch.zeros_like(u_full)
        out["g_D"] = torch.where(bm, u_full, zero)
        out["lap_gD"] = torch.where(bm, full(lu), zero)
        out["bilap"] = torch.where(bm, full(l2u), zero)
    out["u_exact"] = u_full
    gN, gNN, lw = [], [], []
    for a in range(dim):
        tang = [v for b, v in enumerate(xs) if b != a]
        lt = lambda e: sum(sp.diff(e, v, 2) for v in tang)  # noqa: E731
        unn = sp.diff(u, xs[a], 2)
        w = 2 * lt(unn) + lt(lt(u))
        for side in (0, 1):
            pc = face_coords(N, lo, hi, a, side)

            def ev(e):
                return np.broadcast_to(np.asarray(_lamb(e, dim, "numpy")(*pc), dtype=float), pc[0].shape).copy()
            du = ev(sp.diff(u, xs[a]))
            gN.append(-du if side == 0 else du)
            gNN.append(ev(unn))
            lw.append(ev(w))
    for key, arr in (("g_N", gN), ("g_NN", gNN), ("lapt_w", lw)):
        v = np.concatenate(arr)
        out[key] = v if backend == "numpy" else _to_t(v, device)
    return out


# ----------------------------------------------------------------------------
# serving workload: a seeded stream of requests with closed-form data
# ----------------------------------------------------------------------------
#
# Request r (r = 0, 1, ...) draws its grid, its coefficient and its exact
# solution from numpy's default_rng(seed) stream (the shape mix) and from its
# own id (the coefficient: the Fourier recipe above with M = 6, K = 4, A = 0.5
# and seed r):
#   * dim 2 with probability 0.7, N uniform in {128, 256, 512, 1024, 2048};
#     dim 3 otherwise, N uniform in {64, 128, 256};
#   * u = prod_a sin^2(pi x_a) cos(m_a pi x_a), m_a uniform in {0, ..., 4};
#   * arrivals: a Poisson process (exponential gaps) of the given rate.
# u vanishes with its normal derivative on every face, and alpha * Laplace u
# vanishes on every edge, so all boundary data are zero; f is
# -Laplace(alpha Laplace u) = -(alpha Lap^2 u + 2 grad alpha . grad Lap u +
# Lap alpha Lap u), evaluated from closed-form derivatives (no symbolic work
# per request).

SERVE_2D = (128, 256, 512, 1024, 2048)
SERVE_3D = (64, 128, 256)


@dataclass
class RequestSpec:
    rid: int
    dim: int
    N: int
    m: Tuple[int, ...]
    arrival: float  # seconds from the start of the stream
    deadline: Optional[float] = None  # seconds from the start of the stream; None: no deadline


def request_stream(n: int, rate: float, seed: int = 5, p2d: float = 0.7,
                   sizes2d: Sequence[int] = SERVE_2D, sizes3d: Sequence[int] = SERVE_3D) -> List[RequestSpec]:
    """n requests with Poisson arrivals of `rate` per second."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(n):
        t += rng.exponential(1.0 / rate) if rate > 0 else 0.0
        if rng.uniform() < p2d:
            dim, N = 2, int(rng.choice(sizes2d))
        else:
            dim, N = 3, int(rng.choice(sizes3d))
        m = tuple(int(v) for v in rng.integers(0, 5, size=dim))
        out.append(RequestSpec(r, dim, N, m, t))
    return out


def _cos_terms(m: int):
    """sin^2(pi x) cos(m pi x) as a sum of a_j cos(w_j x)."""
    return [(0.5, m * math.pi), (-0.25, (m + 2) * math.pi), (-0.25, (m - 2) * math.pi)]


def _g_derivs(x, m: int):
    """g, g', g'', g''', g'''' of g(x) = sin^2(pi x) cos(m pi x) at x (torch)."""
    import torch
    out = [torch.zeros_like(x) for _ in range(5)]
    for a, w in _cos_terms(m):
        c, s = torch.cos(w * x), torch.sin(w * x)
        out[0] += a * c
        out[1] += -a * w * s
        out[2] += -a * w ** 2 * c
        out[3] += a * w ** 3 * s
        out[4] += a * w ** 4 * c
    return out


_ALPHA_MAX: Dict[Tuple[int, int], float] = {}


def _alpha_norm(dim: int, modes, device) -> float:
    import torch
    L = 1024 if dim == 2 else 128
    t = torch.linspace(0.0, 1.0, L + 1, dtype=torch.float64, device=device)
    grids = torch.meshgrid(*([t] * dim), indexing="ij")
    val = torch.zeros_like(grids[0])
    for k, c, th in modes:
        val += c * torch.cos(2 * math.pi * sum(k[a] * grids[a] for a in range(dim)) + th)
    return float(val.abs().max())


def exact_request(spec: RequestSpec, device="cuda"):
    """The exact u of a request on its full grid (flat float64 tensor)."""
    import torch
    dim, N = spec.dim, spec.N
    x = torch.arange(N + 1, dtype=torch.float64, device=device) / N
    out = None
    for a in range(dim):
        shp = [1] * dim
        shp[dim - 1 - a] = N + 1
        g = _g_derivs(x, spec.m[a])[0].reshape(shp)
        out = g if out is None else out * g
    return out.expand((N + 1,) * dim).reshape(-1).contiguous()


def request_numpy(spec: RequestSpec) -> Dict[str, object]:
    """A request's alpha, f and exact u on the host (numpy, full-grid shape
    reversed as ``sample`` returns it; every boundary datum of a request is
    zero), for the CPU oracle."""
    d = sample_request(spec, device="cpu", with_exact=True)
    shape = (spec.N + 1,) * spec.dim
    out = {k: d[k] for k in ("dim", "N", "lo", "hi", "name")}
    for k in ("alpha", "f", "u_exact"):
        out[k] = d[k].numpy().reshape(shape)
    return out


def sample_request(spec: RequestSpec, device="cuda", out_alpha=None, out_f=None, with_exact: bool = False,
                   M: int = 6, K: int = 4, A: float = 0.5) -> Dict[str, object]:
    """alpha and f of a request on its full grid (float64 tensors on device);
    written into out_alpha / out_f (flat views) when given."""
    import torch
    dim, N = spec.dim, spec.N
    modes = fourier_modes(dim, M, K, spec.rid)
    mx = _alpha_norm(dim, modes, device)
    x = torch.arange(N + 1, dtype=torch.float64, device=device) / N
    g = [_g_derivs(x, spec.m[a]) for a in range(dim)]

    def axis(v, a):  # 1D array along axis a of the (reversed) full-grid shape
        shp = [1] * dim
        shp[dim - 1 - a] = N + 1
        return v.reshape(shp)

    G = [[axis(g[a][k], a) for k in range(5)] for a in range(dim)]
    shape = (N + 1,) * dim

    def prod(parts):
        out = parts[0]
        for q in parts[1:]:
            out = out * q
        return out.expand(shape) if out.shape != shape else out

    # alpha and its derivatives
    al = torch.ones(shape, dtype=torch.float64, device=device)
    dal = [torch.zeros(shape, dtype=torch.float64, device=device) for _ in range(dim)]
    lal = torch.zeros(shape, dtype=torch.float64, device=device)
    X_ = [axis(x, a) for a in range(dim)]
    for k, c, th in modes:
        ph = 2 * math.pi * sum(k[a] * X_[a] for a in range(dim)) + th
        cph, sph = torch.cos(ph), torch.sin(ph)
        s = A * c / mx
        al = al + s * cph
        for a in range(dim):
            dal[a] = dal[a] - s * 2 * math.pi * k[a] * sph
        lal = lal - s * (2 * math.pi) ** 2 * sum(kk * kk for kk in k) * cph
    # Laplace u, its gradient and the bi-Laplacian of the separable u
    def term(sel):  # product over axes of G[a][sel[a]]
        return prod([G[a][sel[a]] for a in range(dim)])
    lap = sum(term([2 if b == a else 0 for b in range(dim)]) for a in range(dim))
    glap = []
    for c in range(dim):
        acc = 0
        for a in range(dim):
            sel = [2 if b == a else 0 for b in range(dim)]
            sel[c] += 1
            acc = acc + term(sel)
        glap.append(acc)
    bil = 0
    for a in range(dim):
        for c in range(dim):
            sel = [0] * dim
            sel[a] += 2
            sel[c] += 2
            bil = bil + term(sel)
    f = -(al * bil + 2 * sum(dal[c] * glap[c] for c in range(dim)) + lal * lap)
    res: Dict[str, object] = {"dim": dim, "N": [N] * dim, "lo": (0.0,) * dim, "hi": (1.0,) * dim,
                              "name": "request%d" % spec.rid}
    if out_alpha is not None:
        out_alpha.copy_(al.reshape(-1))
        res["alpha"] = out_alpha
    else:
        res["alpha"] = al.reshape(-1).contiguous()
    if out_f is not None:
        out_f.copy_(f.reshape(-1))
        res["f"] = out_f
    else:
        res["f"] = f.reshape(-1).contiguous()
    if with_exact:
        res["u_exact"] = term([0] * dim).reshape(-1).contiguous()
    return res
