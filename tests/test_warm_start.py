"""GMRES from the caller's initial Q (``ahoc_solve_from``): the same discrete
solution as a cold start, no iteration from a converged Q, and the per-problem
rules of a batch (zero data keeps Q = 0, a non-finite guess fails its problem
alone)."""

import numpy as np
import pytest
import torch

from oracle import coupled
from paper_2609_16478_b300 import ahoc, inputs

pytestmark = pytest.mark.gpu

TOL_SOLVE = 1e-10


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).reshape(-1).cuda()


def _rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_converged_q_takes_no_iteration():
    """Restarting from the converged Q of the same problem: zero GMRES
    iterations, no coarse level, and the same u."""
    d = inputs.sample(inputs.config_problem("fourier2d"), [256, 256])
    p = ahoc.plan_for(d)
    f = _dev(d["f"])
    u1, i1 = p.solve(f, tol=1e-12)
    q, _ = p.last_qv(with_v=False)
    u2, i2 = p.solve(f, tol=1e-12, q0=q.clone())
    assert i2["iters"] == 0 and i2["levels"] == 0, i2
    assert i2["rel_resid"] <= 1e-12
    assert _rel(u2.cpu().numpy(), u1.cpu().numpy()) < 1e-12
    p.close()


@pytest.mark.parametrize("name,N", [("sincos2d", [64, 64]), ("sincos3d", [16, 16, 16]), ("navier2d", [64, 64])])
def test_random_guess_gives_the_oracle_solution(name, N):
    """From a random Q the solve reaches the oracle's direct solution of the
    coupled system (nonzero boundary data of every kind; 2D, fused 3D, Navier)."""
    d = inputs.sample(inputs.config_problem(name), N)
    ref = coupled.solve_direct(coupled.assemble(d), d)
    p = ahoc.plan_for(d)
    q0 = torch.randn(p.ngamma, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    u, info = p.solve(_dev(d["f"]), tol=1e-13, q0=q0)
    assert info["iters"] > 0
    U = u.cpu().numpy().reshape(tuple(n + 1 for n in reversed(N)))
    assert _rel(U, ref.U) < TOL_SOLVE
    p.close()


def test_batch_zero_data_and_nonfinite_guess():
    """A batch of three: problem 0 from a random guess equals its cold solve;
    problem 1 has zero data, so its Q and u are 0 whatever its guess; problem
    2's guess holds a NaN, so it alone fails (AHOC_ENUMERIC)."""
    dim, N, B = 2, 64, 3
    specs = [inputs.RequestSpec(r, dim, N, (1, 2), 0.0) for r in range(B)]
    ds = [inputs.sample_request(s, device="cuda") for s in specs]
    ds[1]["f"] = torch.zeros_like(ds[1]["f"])
    nf = (N + 1) ** dim
    pb = ahoc.Plan(dim, [N] * dim, torch.cat([d["alpha"] for d in ds]), batch=B)
    ng = pb.ngamma
    q0 = torch.randn(B * ng, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(4))
    q0[2 * ng + 5] = float("nan")
    ub, infos = pb.solve(torch.cat([d["f"] for d in ds]), tol=1e-12, q0=q0, check=False)
    assert infos[2]["status"] == ahoc.AHOC_ENUMERIC
    assert infos[0]["status"] == ahoc.AHOC_OK and infos[1]["status"] == ahoc.AHOC_OK
    qb, _ = pb.last_qv(with_v=False)
    assert float(qb[ng:2 * ng].abs().max()) == 0.0
    assert float(ub[nf:2 * nf].abs().max()) == 0.0
    ps = ahoc.Plan(dim, [N] * dim, ds[0]["alpha"])
    us, _ = ps.solve(ds[0]["f"], tol=1e-12)
    assert _rel(ub[:nf].cpu().numpy(), us.cpu().numpy()) < TOL_SOLVE
    pb.close()
    ps.close()


def test_mixed_plan_refuses_a_guess():
    d = inputs.sample(inputs.config_problem("smooth2d"), [64, 64])
    p = ahoc.plan_for(d, prec="mixed")
    q0 = torch.zeros(p.ngamma, dtype=torch.float64, device="cuda")
    with pytest.raises(ahoc.AhocError, match="EUNSUPPORTED"):
        p.solve(_dev(d["f"]), tol=1e-12, q0=q0)
    p.close()


def test_nested_guess_batch_with_a_zero_data_problem():
    """The nested coarse-grid guess in a batch where one problem's data are
    zero: GMRES leaves that problem alone (b = 0), and its u is exactly 0
    even after an earlier solve left other values in the plan's buffers."""
    dim, N, B = 2, 64, 2
    specs = [inputs.RequestSpec(r, dim, N, (2, 1), 0.0) for r in range(B)]
    ds = [inputs.sample_request(s, device="cuda") for s in specs]
    nf = (N + 1) ** dim
    pb = ahoc.Plan(dim, [N] * dim, torch.cat([d["alpha"] for d in ds]), batch=B, levels=1)
    f = torch.cat([d["f"] for d in ds])
    u_first, _ = pb.solve(f, tol=1e-12)
    assert float(u_first[nf:].abs().max()) > 0
    f[nf:] = 0.0
    ub, infos = pb.solve(f, tol=1e-12)
    assert float(ub[nf:].abs().max()) == 0.0
    ps = ahoc.Plan(dim, [N] * dim, ds[0]["alpha"], levels=1)
    us, _ = ps.solve(ds[0]["f"], tol=1e-12)
    assert torch.equal(ub[:nf], us)
    pb.close()
    ps.close()
