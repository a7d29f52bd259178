"""Batched plans: every problem of a batch gives the bits of its own solve.

A batched plan runs each launch over all its problems and GMRES in
lockstep, masking converged problems out; the per-problem arithmetic --
including the block split of every reduction -- does not depend on the
batch, so results, iteration counts and residuals must be identical to a
single-problem plan's.
"""

import numpy as np
import pytest
import torch

from oracle import coupled
from paper_2609_16478_b300 import ahoc, inputs

pytestmark = pytest.mark.gpu

MS = {2: [(3, 1), (0, 4), (2, 2)], 3: [(0, 4, 2), (1, 1, 3), (4, 0, 0)]}


def _requests(dim, N, B, first=0):
    specs = [inputs.RequestSpec(first + r, dim, N, MS[dim][r % 3], 0.0) for r in range(B)]
    return [inputs.sample_request(s, device="cuda") for s in specs]


def _solo(d, prec, **kw):
    p = ahoc.Plan(d["dim"], d["N"], d["alpha"], prec=prec, **kw)
    u, info = p.solve(d["f"], tol=1e-12)
    return p, u, info


@pytest.mark.parametrize("dim,N,prec", [(2, 64, "fp64"), (2, 256, "fp64"), (2, 128, "mixed"), (3, 16, "fp64"),
                                        (3, 32, "mixed"), (3, 128, "fp64")])
def test_batch_equals_solo(dim, N, prec):
    B = 3
    ds = _requests(dim, N, B)
    nf = (N + 1) ** dim
    pb = ahoc.Plan(dim, [N] * dim, torch.cat([d["alpha"] for d in ds]), prec=prec, batch=B)
    ub, infos = pb.solve(torch.cat([d["f"] for d in ds]), tol=1e-12)
    qb, _ = pb.last_qv(with_v=False)
    for b in range(B):
        ps, us, info = _solo(ds[b], prec)
        assert torch.equal(ub[b * nf:(b + 1) * nf], us), b
        assert infos[b]["iters"] == info["iters"] and infos[b]["rel_resid"] == info["rel_resid"]
        assert infos[b]["coarse_iters"] == info["coarse_iters"]
        assert infos[b]["refine_steps"] == info["refine_steps"]
        q, _ = ps.last_qv(with_v=False)
        assert torch.equal(qb[b * pb.ngamma:(b + 1) * pb.ngamma], q)


@pytest.mark.parametrize("dim,N,prec", [(2, 64, "fp64"), (2, 64, "mixed"), (3, 16, "fp64"), (3, 16, "mixed")])
def test_batch_matches_oracle(dim, N, prec):
    """Every problem of a batched solve against the CPU oracle's direct solve
    of the same request (relative L2 on the full grid)."""
    B = 3
    specs = [inputs.RequestSpec(r, dim, N, MS[dim][r % 3], 0.0) for r in range(B)]
    ds = [inputs.sample_request(s, device="cuda") for s in specs]
    nf = (N + 1) ** dim
    pb = ahoc.Plan(dim, [N] * dim, torch.cat([d["alpha"] for d in ds]), prec=prec, batch=B)
    ub, infos = pb.solve(torch.cat([d["f"] for d in ds]), tol=1e-12)
    for b, s in enumerate(specs):
        h = inputs.request_numpy(s)
        sol = coupled.solve_direct(coupled.assemble(h), h)
        u = ub[b * nf:(b + 1) * nf].cpu().numpy().reshape(sol.U.shape)
        rel = np.linalg.norm(u - sol.U) / np.linalg.norm(sol.U)
        assert rel < (1e-10 if prec == "fp64" else 1e-9), (b, rel, infos[b])


@pytest.mark.parametrize("dim,N,prec", [(2, 128, "fp64"), (3, 32, "mixed")])
def test_mask_and_reload(dim, N, prec):
    B = 3
    ds = _requests(dim, N, B)
    nf = (N + 1) ** dim
    pb = ahoc.Plan(dim, [N] * dim, torch.cat([d["alpha"] for d in ds]), prec=prec, batch=B)
    f = torch.cat([d["f"] for d in ds])
    # problem 1 sits out: its output is untouched, the others are their own solves
    pb.set_active([1, 0, 1])
    u = torch.full((B * nf,), 7.0, dtype=torch.float64, device="cuda")
    _, infos = pb.solve(f, u, tol=1e-12)
    assert infos[1] is None
    assert torch.all(u[nf:2 * nf] == 7.0)
    for b in (0, 2):
        _, us, _ = _solo(ds[b], prec)
        assert torch.equal(u[b * nf:(b + 1) * nf], us)
    # a new problem in slot 1, all three taking part
    new = _requests(dim, N, 1, first=40)[0]
    pb.load(1, new["alpha"])
    f[nf:2 * nf] = new["f"]
    pb.set_active([1, 1, 1])
    u, infos = pb.solve(f, tol=1e-12)
    _, us, info = _solo(new, prec)
    assert torch.equal(u[nf:2 * nf], us) and infos[1]["iters"] == info["iters"]


def test_batched_matvec_and_rhs():
    dim, N, B = 2, 64, 4
    ds = _requests(dim, N, B)
    pb = ahoc.Plan(dim, [N] * dim, torch.cat([d["alpha"] for d in ds]), batch=B)
    q = torch.randn(B * pb.ngamma, dtype=torch.float64, device="cuda",
                    generator=torch.Generator("cuda").manual_seed(3))
    y = pb.matvec(q)
    b = pb.schur_rhs(torch.cat([d["f"] for d in ds]))
    n = pb.ngamma
    for i in range(B):
        ps = ahoc.Plan(dim, [N] * dim, ds[i]["alpha"])
        assert torch.equal(y[i * n:(i + 1) * n], ps.matvec(q[i * n:(i + 1) * n].contiguous()))
        assert torch.equal(b[i * n:(i + 1) * n], ps.schur_rhs(ds[i]["f"]))
