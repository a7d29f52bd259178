"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: the FP64 path must match the oracle's direct solve to relative
L2 <= 1e-10 on U (the method reaches the same discrete solution up to the
GMRES tolerance 1e-12 times the Schur condition number); component kernels
(DST, Poisson, Schur action) are held to 1e-12 relative.
"""

import math

import numpy as np
import pytest
import torch

from conftest import golden
from oracle import coupled, dst, residual
from paper_2609_16478_b300 import ahoc, inputs

pytestmark = pytest.mark.gpu

TOL_SOLVE = 1e-10
TOL_COMP = 1e-12


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).reshape(-1).cuda()


def _host(t, shape):
    return t.detach().cpu().numpy().reshape(shape)


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def _plan(data, **kw):
    return ahoc.plan_for(data, **kw)


def _blank(N, dim, lo=None, hi=None):
    shape = tuple(n + 1 for n in reversed(N))
    return dict(dim=dim, N=list(N), lo=lo or [0.0] * dim, hi=hi or [1.0] * dim, alpha=np.ones(shape))


# --- component kernels --------------------------------------------------------

@pytest.mark.parametrize("radix", [4, 8])
@pytest.mark.parametrize("N,axis", [((8, 8), 0), ((64, 64), 0), ((4096, 16), 0), ((32, 16), 0), ((2048, 8), 0),
                                    ((16, 32, 8), 0), ((16, 32, 8), 1), ((8, 1024, 8), 1), ((128, 64, 16), 1),
                                    ((256, 512, 8), 1)])
def test_dst1_matches_definition(N, axis, radix):
    """DST-I along x and y against the definition (scipy), radix-4 and
    radix-8 stages (the tuner's choice); the sizes cover each stage plan:
    log2(N/2) = 0, 1, 2 mod 3 (radix-8: a radix-8 run, a radix-2 or a radix-4
    stage first) and even and odd (radix-4: a radix-2 stage first)."""
    dim = len(N)
    L = ahoc.lib()
    L.ahoc_tune_set(ahoc.AHOC_TUNE_DST_RADIX, dim, N[0], ahoc.AHOC_FP64, radix)
    try:
        p = _plan(_blank(N, dim))
    finally:
        L.ahoc_tune_set(ahoc.AHOC_TUNE_DST_RADIX, dim, N[0], ahoc.AHOC_FP64, 0)
    rng = np.random.default_rng(7)
    shape = tuple(n - 1 for n in reversed(N))
    x = rng.normal(size=shape)
    y = _host(p.dst1(_dev(x), axis), shape)
    ref = dst.dst1(x, axis=dim - 1 - axis)
    assert _rel(y, ref) < TOL_COMP * math.log2(N[axis])


@pytest.mark.parametrize("N,lo,hi", [((64, 64), None, None), ((32, 16), [0, -0.5], [1, 0.3]), ((8, 8), None, None),
                                     ((16, 16, 8), None, None), ((8, 16, 32), [0, 0, 0], [1, 2, 0.5])])
def test_poisson_matches_sparse_solve(N, lo, hi):
    dim = len(N)
    p = _plan(_blank(N, dim, lo, hi))
    rng = np.random.default_rng(3)
    shape = tuple(n - 1 for n in reversed(N))
    r = rng.normal(size=shape)
    w = _host(p.poisson(_dev(r)), shape)
    ref = coupled.poisson_solve(N, r, lo, hi)
    assert _rel(w, ref) < TOL_COMP * 10


# --- Lemma 1: the Schur action and right-hand side ---------------------------

@pytest.mark.parametrize("name,N,fused", [("sincos2d", [8, 8], True), ("smooth2d", [16, 16], True),
                                          ("sincos2d", [16, 8], True), ("sincos3d", [8, 8, 8], True),
                                          ("fourier3d", [8, 16, 8], True), ("sincos3d", [8, 8, 8], False),
                                          ("fourier3d", [16, 8, 8], True), ("fourier3d", [16, 8, 8], False)])
def test_schur_matrix_columns(name, N, fused):
    """Columns of ahoc_matvec against the oracle's explicit Schur complement
    (3D: the fused four-pass matvec and the plain one)."""
    prob = inputs.config_problem(name)
    d = inputs.sample(prob, N)
    p = _plan(d, fused=fused)
    B = coupled.Blocks(coupled.assemble(d))
    S = B.schur_dense()
    ng = p.ngamma
    Sg = np.empty((ng, ng))
    e = torch.zeros(ng, dtype=torch.float64, device="cuda")
    for j in range(ng):
        e.zero_()
        e[j] = 1.0
        Sg[:, j] = p.matvec(e).cpu().numpy()
    assert _rel(Sg, S) < TOL_COMP * 10
    b = p.schur_rhs(_dev(d["f"])).cpu().numpy()
    assert _rel(b, B.schur_rhs()) < TOL_COMP * 10


# --- full solves against the direct solve -------------------------------------

@pytest.mark.parametrize("name,N,lo,hi", [
    ("smooth2d", [64, 64], None, None),          # the small configuration, GMRES tol 1e-12
    ("sincos2d", [32, 32], None, None),         # nonzero g_D, g_N, tangential Laplacian, corner v
    ("sincos2d", [64, 16], (0.0, -0.2), (1.0, 0.4)),   # anisotropic box and grid
    ("fourier2d", [128, 128], None, None),
    ("cavity", [64, 64], None, None),
    ("plate", [64, 64], None, None),
    ("sincos3d", [16, 16, 16], None, None),
    ("fourier3d", [16, 8, 16], None, None),
    ("poly2d", [8, 8], None, None),             # smallest grid
])
def test_solve_matches_oracle(name, N, lo, hi):
    prob = inputs.config_problem(name)
    d = inputs.sample(prob, N, lo=lo, hi=hi)
    sol = coupled.solve_direct(coupled.assemble(d), d)
    p = _plan(d)
    u, info = p.solve(_dev(d["f"]), tol=1e-12)
    shape = tuple(n + 1 for n in reversed(N))
    U = _host(u, shape)
    inner = tuple(slice(1, -1) for _ in N)
    assert _rel(U[inner], sol.U[inner]) < TOL_SOLVE, info
    # boundary entries are g_D exactly
    Ub = U.copy()
    Ub[inner] = 0
    Gb = np.asarray(d["g_D"]).reshape(shape).copy()
    Gb[inner] = 0
    assert np.array_equal(Ub, Gb)
    q, v = p.last_qv()
    assert _rel(q.cpu().numpy(), sol.Q) < 1e-9
    assert _rel(_host(v, shape), sol.V) < 1e-9
    assert info["iters"] >= 1 and info["rel_resid"] <= 1e-12


def test_ragged_box_and_minimum_grid():
    """Unequal N per axis (a ragged tail of tiles) and the smallest grid N = 8."""
    for N in ([8, 8, 8], [64, 8], [8, 256]):
        prob = inputs.config_problem("sincos3d" if len(N) == 3 else "sincos2d")
        d = inputs.sample(prob, N)
        sol = coupled.solve_direct(coupled.assemble(d), d)
        u, _ = _plan(d).solve(_dev(d["f"]), tol=1e-12)
        shape = tuple(n + 1 for n in reversed(N))
        assert _rel(_host(u, shape), sol.U) < TOL_SOLVE


def test_zero_data_gives_zero():
    d = inputs.sample(inputs.config_problem("cavity"), [32, 32])
    d["g_N"] = np.zeros_like(d["g_N"])
    u, info = _plan(d).solve(_dev(d["f"]), tol=1e-12)
    assert float(u.abs().max()) == 0.0 and info["iters"] == 0


# --- the paper's printed benchmark values through the CUDA path ----------------

def test_cavity_table6_n1024():
    """Max |U| of the lid-driven cavity at N=1024 equals the paper's Table 6 value."""
    rows = golden("cavity_table6.txt")
    N = int(rows[0][0])
    d = inputs.sample(inputs.config_problem("cavity"), [N, N])
    u, info = _plan(d).solve(_dev(d["f"]), tol=1e-13)
    U = _host(u, (N + 1, N + 1))
    k = np.unravel_index(np.argmax(np.abs(U)), U.shape)
    assert abs(abs(U[k]) - float(rows[0][1])) < 2e-10
    assert abs(k[1] / N - 0.5) < 1e-12 and abs(k[0] / N - float(rows[0][3])) < 1e-4


def test_plate_point_load():
    ref = {r[0]: float(r[1]) for r in golden("plate_sec4.txt")}
    N = 1024
    d = inputs.sample(inputs.config_problem("plate"), [N, N])
    p = _plan(d)
    u, _ = p.solve(_dev(d["f"]), tol=1e-13)
    U = _host(u, (N + 1, N + 1))
    _, v = p.last_qv()
    V = _host(v, (N + 1, N + 1))
    assert abs(U[N // 2, N // 2] - ref["U_center"]) / ref["U_center"] < 2e-4
    assert abs(-V[N, N // 2] - ref["minus_V_top_mid"]) / abs(ref["minus_V_top_mid"]) < 2e-4


# --- full-size configurations: properties that hold at any size ---------------

# error bounds against the exact u: fourth-order estimates from the measured
# errors (2D 4096^2 4.7e-11; 3D 256^3 6.5e-9; the high-wavenumber u at 1024^3
# 1.81e-6, so about 256 times that at 256^3), with a margin
@pytest.mark.parametrize("name,N,prec,err_max", [
    ("fourier2d", [4096, 4096], "fp64", 1e-8), ("fourier2d", [4096, 4096], "mixed", 1e-8),
    ("fourier3d", [128, 128, 128], "fp64", 1e-6), ("fourier3d", [256, 256, 256], "fp64", 1e-7),
    ("fourier3d", [256, 256, 256], "mixed", 1e-7), ("fourier3d_k32", [256, 256, 256], "fp64", 1e-3),
    ("fourier3d_k32", [256, 256, 256], "mixed", 1e-3)])
def test_large_grid_certificate(name, N, prec, err_max):
    """Beyond the direct solver's reach: the oracle's residual certificate of the
    coupled equations evaluated on the GPU solution, and fourth-order accuracy."""
    prob = inputs.config_problem(name)
    dd = inputs.sample(prob, N, backend="torch", device="cuda")
    p = _plan(dd, prec=prec)
    u, info = p.solve(dd["f"].reshape(-1).contiguous(), tol=1e-12)
    shape = tuple(n + 1 for n in reversed(N))
    d = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in dd.items()}
    U = _host(u, shape)
    _, v = p.last_qv()
    V = _host(v, shape)
    ru, rv, rq = residual.coupled_residual(U, V, d)
    # normwise backward errors of the three block rows: |residual| over the
    # sizes of the terms that produce it (||L_h|| |U| etc.); at N = 4096 the
    # 1/h^2 of the stencils turns last-bit differences of U into residuals of
    # ~1e-6 absolute, so only the relative measure is meaningful
    h = [1.0 / n for n in N]
    nL = sum(4.0 / hh ** 2 for hh in h) * (1.0 if len(N) == 2 else 1.5)   # >= ||L_h||_inf / 2
    nD = 12.5 / min(h) ** 2
    amax = np.max(np.abs(d["alpha"]))
    eta_u = np.max(np.abs(ru)) / (nL * np.max(np.abs(U)) + np.max(np.abs(V)) / np.min(np.abs(d["alpha"])))
    eta_v = np.max(np.abs(rv)) / (nL * np.max(np.abs(V)) + np.max(np.abs(d["f"])))
    eta_q = np.max(np.abs(rq)) / (amax * nD * np.max(np.abs(U)) + np.max(np.abs(V)))
    assert max(eta_u, eta_v, eta_q) < 1e-12, (eta_u, eta_v, eta_q)
    err = np.max(np.abs(U - d["u_exact"]))
    assert err < err_max, err
    p.close()


# --- boundary-symbol preconditioner and the tridiagonal paths ------------------

@pytest.mark.parametrize("name,N", [("fourier2d", [256, 256]), ("cavity", [128, 128]), ("sincos3d", [16, 16, 16])])
def test_preconditioner_same_solution_fewer_iterations(name, N):
    d = inputs.sample(inputs.config_problem(name), N)
    f = _dev(d["f"])
    u0, i0 = _plan(d, precond=0).solve(f, tol=1e-12)
    u1, i1 = _plan(d, precond=1).solve(f, tol=1e-12)
    assert _rel(u1.cpu().numpy(), u0.cpu().numpy()) < TOL_SOLVE
    assert i1["iters"] < i0["iters"], (i0["iters"], i1["iters"])


def test_poisson_residual_sequential_tri_path():
    """3D grid with >= 65536 transverse modes: the one-thread-per-mode
    tridiagonal kernel; checked by the oracle's L_h applied to the result."""
    N = (512, 256, 16)
    p = _plan(_blank(N, 3))
    rng = np.random.default_rng(5)
    shape = tuple(n - 1 for n in reversed(N))
    r = rng.normal(size=shape)
    w = _host(p.poisson(_dev(r)), shape)
    A = coupled.laplacian_matrix(N)
    res = A @ w.reshape(-1) - r.reshape(-1)
    assert np.max(np.abs(res)) < 1e-9 * np.max(np.abs(r)) * (N[0] ** 2 * 1e-4)
    # and the chunked path on a grid just below the switch agrees with the sparse solve
    N2 = (64, 32, 16)
    p2 = _plan(_blank(N2, 3))
    shape2 = tuple(n - 1 for n in reversed(N2))
    r2 = rng.normal(size=shape2)
    assert _rel(_host(p2.poisson(_dev(r2)), shape2), coupled.poisson_solve(N2, r2)) < 1e-11


# --- nested (coarse-to-fine) initial guess --------------------------------------

@pytest.mark.parametrize("name,N,levels", [("fourier2d", [256, 256], 1), ("fourier2d", [256, 256], 3),
                                           ("sincos2d", [64, 16], 1), ("sincos3d", [16, 16, 16], 1),
                                           ("cavity", [64, 64], 2)])
def test_nested_initial_guess_matches_oracle(name, N, levels):
    d = inputs.sample(inputs.config_problem(name), N)
    sol = coupled.solve_direct(coupled.assemble(d), d)
    f = _dev(d["f"])
    u1, i1 = _plan(d, levels=levels).solve(f, tol=1e-12)
    shape = tuple(n + 1 for n in reversed(N))
    assert _rel(_host(u1, shape), sol.U) < TOL_SOLVE, i1
    assert i1["levels"] >= 1 and i1["coarse_iters"] > 0
    u0, i0 = _plan(d, levels=0).solve(f, tol=1e-12)
    assert i0["levels"] == 0
    if name != "cavity":   # smooth data: the interpolated coarse solution saves fine iterations
        assert i1["iters"] < i0["iters"], (i0["iters"], i1["iters"])


def test_nested_guess_skips_unresolved_data():
    """The automatic nested guess uses a coarse level only where the coarse
    grid resolves the data (its Schur right-hand side, doubled on clamped
    faces, within 10 % of the finer one's): the smooth workload keeps its
    levels, the high-wavenumber one (sin(32 pi x) factors, under-resolved at
    128^3) gets none; both solves are the ones without nesting, to GMRES
    accuracy."""
    N = [256, 256, 256]
    for name, want in (("fourier3d", True), ("fourier3d_k32", False)):
        d = inputs.sample(inputs.config_problem(name), N, backend="torch", device="cuda")
        d.pop("v_exact", None)
        f = d["f"].reshape(-1).contiguous()
        u1, i1 = _plan(d).solve(f, tol=1e-12)
        assert (i1["levels"] >= 1) == want, (name, i1["levels"])
        assert (i1["coarse_iters"] > 0) == want
        u0, i0 = _plan(d, levels=0).solve(f, tol=1e-12)
        rel = float(torch.linalg.norm(u1 - u0) / torch.linalg.norm(u0))
        assert rel < TOL_SOLVE, (name, rel)


# --- mixed precision: FP32 inner solves, FP64 iterative refinement -------------

TOL_MIXED = 1e-9


@pytest.mark.parametrize("name,N", [("fourier2d", [256, 256]), ("sincos3d", [32, 32, 32]), ("fourier3d", [32, 32, 32])])
def test_mixed_first_step_fp64_and_fp32_match_oracle(name, N):
    """The first correction's right-hand side and recovery by FP64 solves
    (the default) or FP32 ones (opts.first32): both refined results against
    the oracle, and the FP64 first step brings the Schur residual down by at
    least the FP32 operator's accuracy."""
    d = inputs.sample(inputs.config_problem(name), N)
    sol = coupled.solve_direct(coupled.assemble(d), d)
    f = _dev(d["f"])
    shape = tuple(n + 1 for n in reversed(N))
    u1, i1 = _plan(d, prec="mixed").solve(f, tol=1e-12)
    assert i1["status"] == 0 and _rel(_host(u1, shape), sol.U) < TOL_MIXED, i1
    assert i1["refine_hist"][1] < 1e-3, i1["refine_hist"]
    u0, i0 = _plan(d, prec="mixed", first32=True).solve(f, tol=1e-12)
    assert i0["status"] == 0 and _rel(_host(u0, shape), sol.U) < TOL_MIXED, i0


@pytest.mark.parametrize("name,N,levels", [("fourier2d", [256, 256], 2), ("sincos3d", [32, 32, 32], 1)])
def test_mixed_nested_guess_matches_oracle(name, N, levels):
    """A mixed plan with an explicit nested guess (coarse levels that are
    mixed-precision solves themselves): the refined result against the
    oracle, and the first correction solve shorter than from zero."""
    d = inputs.sample(inputs.config_problem(name), N)
    sol = coupled.solve_direct(coupled.assemble(d), d)
    f = _dev(d["f"])
    shape = tuple(n + 1 for n in reversed(N))
    u1, i1 = _plan(d, prec="mixed", levels=levels).solve(f, tol=1e-12)
    assert _rel(_host(u1, shape), sol.U) < TOL_MIXED, i1
    assert i1["levels"] == levels and i1["coarse_iters"] > 0
    u0, i0 = _plan(d, prec="mixed").solve(f, tol=1e-12)
    assert i0["levels"] == 0 and i0["coarse_iters"] == 0   # automatic: off in a mixed plan
    assert _rel(_host(u0, shape), sol.U) < TOL_MIXED
    assert i1["inner_iters"][0] < i0["inner_iters"][0], (i0["inner_iters"], i1["inner_iters"])


@pytest.mark.parametrize("name,N", [("smooth2d", [64, 64]), ("fourier2d", [256, 256]), ("sincos2d", [32, 32]),
                                    ("cavity", [64, 64]), ("sincos3d", [16, 16, 16]), ("fourier3d", [16, 8, 16]),
                                    ("sincos2d", [64, 16])])
def test_mixed_solve_matches_oracle(name, N):
    d = inputs.sample(inputs.config_problem(name), N)
    sol = coupled.solve_direct(coupled.assemble(d), d)
    p = _plan(d, prec="mixed")
    u, info = p.solve(_dev(d["f"]), tol=1e-12)
    shape = tuple(n + 1 for n in reversed(N))
    assert _rel(_host(u, shape), sol.U) < TOL_MIXED, info
    assert info["refine_steps"] >= 2
    q, v = p.last_qv()
    assert _rel(q.cpu().numpy(), sol.Q) < 1e-8 and _rel(_host(v, shape), sol.V) < 1e-8


@pytest.mark.parametrize("name,N", [("sincos2d", [16, 16]), ("sincos3d", [8, 8, 8])])
def test_mixed_matvec_is_fp32_accurate(name, N):
    d = inputs.sample(inputs.config_problem(name), N)
    p = _plan(d, prec="mixed")
    S = coupled.Blocks(coupled.assemble(d)).schur_dense()
    ng = p.ngamma
    Sg = np.empty((ng, ng))
    e = torch.zeros(ng, dtype=torch.float64, device="cuda")
    for j in range(ng):
        e.zero_()
        e[j] = 1.0
        Sg[:, j] = p.matvec(e).cpu().numpy()
    assert _rel(Sg, S) < 1e-5


def test_mixed_equals_fp64_at_1024():
    d = inputs.sample(inputs.config_problem("fourier2d"), [1024, 1024], backend="torch", device="cuda")
    f = d["f"].reshape(-1).contiguous()
    u64, i64 = _plan(d).solve(f, tol=1e-12)
    umx, imx = _plan(d, prec="mixed").solve(f, tol=1e-12)
    rel = float(torch.linalg.norm(umx - u64) / torch.linalg.norm(u64))
    assert rel < TOL_MIXED, (rel, imx)
    err = float((umx.reshape(1025, 1025) - d["u_exact"]).abs().max())
    err64 = float((u64.reshape(1025, 1025) - d["u_exact"]).abs().max())
    assert err < 1.05 * err64 + 1e-15


def test_mixed_equals_fp64_3d_512():
    # 511^2 transverse modes: the grid on which a column-wise FP32 tridiagonal
    # recurrence stalled the refinement at ~1e-5; the chunked form with FP64
    # carries must take the mixed solve to the FP64 answer
    N = [512, 512, 512]
    d = inputs.sample(inputs.config_problem("fourier3d"), N, backend="torch", device="cuda")
    f = d["f"].reshape(-1).contiguous()
    p64 = _plan(d)
    u64, i64 = p64.solve(f, tol=1e-12)
    p64.close()
    del p64
    pmx = _plan(d, prec="mixed")
    umx, imx = pmx.solve(f, tol=1e-12)
    assert imx["status"] == 0 and imx["refine_steps"] <= 6, imx
    hist = imx["refine_hist"]
    assert all(hist[k + 1] < 0.5 * hist[k] for k in range(imx["refine_steps"]))
    rel = float(torch.linalg.norm(umx - u64) / torch.linalg.norm(u64))
    assert rel < TOL_MIXED, (rel, imx)


def test_mixed_limiting_accuracy_k32():
    # u = prod sin^2(pi x_a) sin(32 pi x_a): v = alpha Laplace u vanishes on every
    # face, so the Schur right-hand side is at discretisation level while the
    # interior fields are O(1e4); the refinement's residual then stops at the
    # floor of its FP64 evaluation, and the solve ends on the size of the last
    # correction.  It must agree with the FP64 solve all the same.
    N = [256, 256, 256]
    d = inputs.sample(inputs.config_problem("fourier3d_k32"), N, backend="torch", device="cuda")
    f = d["f"].reshape(-1).contiguous()
    u64, _ = _plan(d).solve(f, tol=1e-12)
    umx, imx = _plan(d, prec="mixed").solve(f, tol=1e-12)
    assert imx["status"] == 0, imx
    k = imx["refine_steps"]
    assert imx["refine_hist"][k] <= 1e-12 or imx["refine_du"][k - 1] <= 1e-12, imx
    rel = float(torch.linalg.norm(umx - u64) / torch.linalg.norm(u64))
    assert rel < TOL_MIXED, (rel, imx)


def test_mixed_refines_on_at_the_floor():
    # a serving request whose Schur residual stalls just above tol = 1e-12
    # while its corrections still shrink: the refinement must go on and
    # converge (and agree with the FP64 solve)
    spec = inputs.RequestSpec(704, 2, 2048, (4, 2), 0.0)
    d = inputs.sample_request(spec, device="cuda")
    pm = ahoc.Plan(2, [2048, 2048], d["alpha"], prec="mixed", restart=60, max_iters=2000)
    um, im = pm.solve(d["f"], tol=1e-12)
    assert im["status"] == 0, im
    p64 = ahoc.Plan(2, [2048, 2048], d["alpha"], restart=60, max_iters=2000)
    u64, _ = p64.solve(d["f"], tol=1e-12)
    assert float(torch.linalg.norm(um - u64) / torch.linalg.norm(u64)) < TOL_MIXED


# --- host-buffer entry point -----------------------------------------------------

@pytest.mark.parametrize("name,N,prec", [("smooth2d", [64, 64], "fp64"), ("sincos3d", [16, 16, 16], "mixed")])
def test_solve_host_matches_device_solve_and_oracle(name, N, prec):
    """ahoc_solve_host (f and u in host memory, copies on the plan's stream)
    gives the device-pointer solve's result bit for bit, and the oracle's."""
    d = inputs.sample(inputs.config_problem(name), N)
    sol = coupled.solve_direct(coupled.assemble(d), d)
    p = _plan(d, prec=prec)
    f = _dev(d["f"])
    u_dev, _ = p.solve(f, tol=1e-12)
    f_host = torch.as_tensor(np.ascontiguousarray(d["f"]), dtype=torch.float64).reshape(-1).pin_memory()
    u_host = torch.full_like(f_host, float("nan")).pin_memory()
    for _ in range(2):
        p.solve_host(f_host, u_host, tol=1e-12)
        assert torch.equal(u_host, u_dev.cpu())
    shape = tuple(n + 1 for n in reversed(N))
    assert _rel(u_host.numpy().reshape(shape), sol.U) < (TOL_SOLVE if prec == "fp64" else 1e-9)
    p.close()


def test_fused3d_matvec_on_many_modes():
    """A 3D grid with 511 x 255 transverse modes (the one-thread-per-column
    z-solve of the large grids): the fused Schur action equals the plain
    one (checked against the oracle's Schur matrix on small grids above), and
    both are linear in q."""
    N = (512, 256, 8)
    prob = inputs.config_problem("fourier3d")
    d = inputs.sample(prob, list(N), lo=[0, 0, 0], hi=[1.0, 0.5, 1.0 / 64])
    pf, pu = _plan(d, fused=True), _plan(d, fused=False)
    g = torch.Generator("cuda").manual_seed(4)
    q1 = torch.randn(pf.ngamma, dtype=torch.float64, device="cuda", generator=g)
    q2 = torch.randn(pf.ngamma, dtype=torch.float64, device="cuda", generator=g)
    yf, yu = pf.matvec(q1), pu.matvec(q1)
    assert float(torch.linalg.norm(yf - yu) / torch.linalg.norm(yu)) < 1e-12
    y12 = pf.matvec(q1 + 2 * q2)
    lin = pf.matvec(q1) + 2 * pf.matvec(q2)
    assert float(torch.linalg.norm(y12 - lin) / torch.linalg.norm(lin)) < 1e-13


@pytest.mark.parametrize("N", [(512, 512), (2048, 64), (256, 256, 8), (256, 2048, 8), (1024, 512, 8)])
def test_mixed_matvec_matches_fp64_on_long_lines(N):
    """The FP32 Schur action (line DSTs of 256 .. 2048 points along x and,
    in 3D, y) against the FP64 action: FP32-accurate.  The bound is about
    160 FP32 unit roundoffs (1e-5) up to 1024-point lines and grows in
    proportion to the longest line beyond: the transforms' rounding grows
    like log N, the amplification by the tridiagonal solves and the
    one-sided trace like N (2048-point lines measure 1.3e-5)."""
    dim = len(N)
    hi = [n / max(N) for n in N]   # equal spacing on every axis
    prob = inputs.config_problem("fourier3d" if dim == 3 else "fourier2d")
    d = inputs.sample(prob, list(N), lo=[0.0] * dim, hi=hi)
    p64, p32 = _plan(d), _plan(d, prec="mixed")
    g = torch.Generator("cuda").manual_seed(6)
    q = torch.randn(p64.ngamma, dtype=torch.float64, device="cuda", generator=g)
    y64, y32 = p64.matvec(q), p32.matvec(q)
    assert float(torch.linalg.norm(y32 - y64) / torch.linalg.norm(y64)) < 1e-5 * max(1.0, max(N) / 1024)
