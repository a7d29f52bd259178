"""Method variants on the GPU: Navier faces (Eq. 2, Lap u = g_L) and the
constant shift beta / alpha of the v-equation (Sec. 2.2), against the oracle
and against the paper's Table 1 (Example 1)."""

import numpy as np
import pytest
import torch

from conftest import golden
from oracle import coupled
from paper_2609_16478_b300 import ahoc, inputs

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def _solve(d, prec="fp64", tol=1e-12):
    p = ahoc.plan_for(d, prec=prec)
    f = torch.as_tensor(np.ascontiguousarray(d["f"]), dtype=torch.float64).reshape(-1).cuda()
    u, info = p.solve(f, tol=tol)
    shape = tuple(n + 1 for n in reversed(d["N"]))
    return p, u.cpu().numpy().reshape(shape), info


@pytest.mark.parametrize("name,N", [("navier2d", [64, 64]), ("navier2d", [64, 32]), ("shift2d", [64, 64]),
                                    ("singular2d", [64, 64]), ("navier3d", [16, 16, 16]),
                                    ("singular2d_eps1e-5", [128, 128])])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-9)])
def test_variant_solve_matches_oracle(name, N, prec, tol):
    d = inputs.sample(inputs.config_problem(name), N)
    sol = coupled.solve_direct(coupled.assemble(d), d)
    p, U, info = _solve(d, prec)
    assert _rel(U, sol.U) < tol, info
    q, _ = p.last_qv(with_v=False)
    # Q of the eps = 1e-5 boundary-layer problem is conditioned ~30x worse than U
    assert _rel(q.cpu().numpy(), sol.Q) < (1e-7 if "eps1e-5" in name else 1e-8)


@pytest.mark.parametrize("name,N", [("navier2d", [8, 8]), ("shift2d", [8, 8]), ("singular2d", [16, 8]),
                                    ("navier3d", [8, 8, 8])])
def test_variant_schur_columns(name, N):
    """S_h e_j from the GPU matvec against the oracle's explicit Schur
    complement: Navier rows are -I, the shift enters every clamped row."""
    d = inputs.sample(inputs.config_problem(name), N)
    S = coupled.Blocks(coupled.assemble(d)).schur_dense()
    p = ahoc.plan_for(d)
    ng = p.ngamma
    e = torch.zeros(ng, dtype=torch.float64, device="cuda")
    Sg = np.empty((ng, ng))
    for j in range(ng):
        e.zero_()
        e[j] = 1.0
        Sg[:, j] = p.matvec(e).cpu().numpy()
    assert _rel(Sg, S) < 1e-11
    b = p.schur_rhs(torch.as_tensor(np.ascontiguousarray(d["f"]), dtype=torch.float64).reshape(-1).cuda())
    assert _rel(b.cpu().numpy(), coupled.Blocks(coupled.assemble(d)).schur_rhs()) < 1e-11


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_example1_table1(prec):
    """Example 1 (Table 1): the maximum error of U at 256^2 .. 2048^2 for
    eps = 1e-4 and 1e-5 equals the printed values to their three digits.
    At 4096^2 this discretisation's error does not move with the GMRES
    tolerance (4.679e-10 and 4.607e-9 for tol 1e-10 .. 1e-14) while the
    printed values are 4.54e-10 and 4.65e-9: the paper stops GMRES at a
    tolerance proportional to h^3.5 (Sec. 4.1), which at that grid reaches the
    printed digits, so the finest row is held to 4%."""
    for row in golden("singular2d_table1.txt"):
        N = int(row[0])
        bar = 0.006 if N <= 2048 else 0.04
        for col, name in ((1, "singular2d"), (2, "singular2d_eps1e-5")):
            d = inputs.sample(inputs.config_problem(name), [N, N], backend="torch", device="cuda")
            p = ahoc.plan_for(d, prec=prec, restart=100, max_iters=1000)
            u, info = p.solve(d["f"].reshape(-1).contiguous(), tol=1e-12)
            err = float((u.reshape(N + 1, N + 1) - d["u_exact"]).abs().max())
            assert abs(err / float(row[col]) - 1) < bar, (N, name, err, row[col], info["iters"])
            p.close()


# --- variable beta / alpha: BiCGSTAB v-solves (FP64), constant-shift corrections (mixed) ---

@pytest.mark.parametrize("name,N", [("varbeta2d", [64, 64]), ("sincos3d_var_5_1_5", [16, 16, 16]),
                                    ("peak3d_q5_p1", [16, 16, 16])])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-9)])
def test_variable_beta_matches_oracle(name, N, prec, tol):
    d = inputs.sample(inputs.config_problem(name), N)
    sol = coupled.solve_direct(coupled.assemble(d), d)
    p, U, info = _solve(d, prec)
    assert _rel(U, sol.U) < tol, info
    if prec == "fp64":
        assert info["vsolve_iters"] > 0


@pytest.mark.parametrize("name,N", [("varbeta2d", [8, 8]), ("sincos3d_var_5_1_5", [8, 8, 8])])
def test_variable_beta_schur_columns(name, N):
    d = inputs.sample(inputs.config_problem(name), N)
    B = coupled.Blocks(coupled.assemble(d))
    S = B.schur_dense()
    p = ahoc.plan_for(d)
    ng = p.ngamma
    e = torch.zeros(ng, dtype=torch.float64, device="cuda")
    Sg = np.empty((ng, ng))
    for j in range(ng):
        e.zero_()
        e[j] = 1.0
        Sg[:, j] = p.matvec(e).cpu().numpy()
    assert _rel(Sg, S) < 1e-11
    b = p.schur_rhs(torch.as_tensor(np.ascontiguousarray(d["f"]), dtype=torch.float64).reshape(-1).cuda())
    assert _rel(b.cpu().numpy(), B.schur_rhs()) < 1e-11


@pytest.mark.parametrize("prec,nmax", [("fp64", 512), ("mixed", 128)])
def test_examples2_3_tables(prec, nmax):
    """Tables 2-3 (Examples 2-3): the maximum error of U at 32^3 .. 256^3
    equals the printed values to their three digits; at 512^3 (the paper's
    GMRES stops at a tolerance proportional to h^3.5, Sec. 4.1) within 1%."""
    names = ["peak3d_q10_p0.2", "peak3d_q5_p1", "sincos3d_var_5_1_5", "sincos3d_var_25_5_25"]
    for row in golden("varbeta3d_tables23.txt"):
        N = int(row[0])
        if N > nmax:
            continue
        for col, name in enumerate(names, start=1):
            d = inputs.sample(inputs.config_problem(name), [N] * 3, backend="torch", device="cuda")
            p = ahoc.plan_for(d, prec=prec, restart=100, max_iters=1000)
            u, info = p.solve(d["f"].reshape(-1).contiguous(), tol=1e-12)
            err = float((u.reshape(N + 1, N + 1, N + 1) - d["u_exact"]).abs().max())
            assert abs(err / float(row[col]) - 1) < (0.006 if N <= 256 else 0.01), (N, name, err, row[col], info["iters"])
            p.close()


@pytest.mark.parametrize("name,N,variable", [("shift2d", [32, 32], False), ("singular2d", [32, 32], False),
                                             ("varbeta2d", [32, 32], True)])
def test_auto_shift_picks_the_beta_class(name, N, variable):
    """opts.auto_shift: the plan reads beta / alpha and chooses the constant
    shift (FFT v-solves only) or variable beta (BiCGSTAB v-solves)."""
    d = inputs.sample(inputs.config_problem(name), N)
    sol = coupled.solve_direct(coupled.assemble(d), d)
    p = ahoc.plan_for(d)
    u, info = p.solve(torch.as_tensor(d["f"]).reshape(-1).contiguous().cuda(), tol=1e-12)
    assert (info["vsolve_iters"] > 0) == variable, info["vsolve_iters"]
    U = u.cpu().numpy().reshape(sol.U.shape)
    assert np.linalg.norm(U - sol.U) / np.linalg.norm(sol.U) < 1e-10
