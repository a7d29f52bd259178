"""The triharmonic class on the GPU (Sec. 4.2, "Triharmonic equation",
Table 5) against the triharmonic oracle: Schur columns and right-hand side,
full solves, and the printed Table 5 errors."""

import numpy as np
import pytest
import torch

from conftest import golden
from oracle import triharmonic as T
from paper_2609_16478_b300 import ahoc, inputs

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def _sample(name, N):
    return inputs.sample_triharmonic(inputs.triharmonic_problem(name), N)


@pytest.mark.parametrize("name,N", [("trisin2d", [8, 8]), ("tripoly2d", [16, 8]), ("tri3d_5_1_5", [8, 8, 8]),
                                    ("tripoly3d", [8, 16, 8])])
def test_tri_schur_columns_and_rhs(name, N):
    d = _sample(name, N)
    B = T.TriBlocks(T.assemble(d))
    S = B.schur_dense()
    p = ahoc.plan_for_triharmonic(d)
    ng = p.ngamma
    Sg = np.empty((ng, ng))
    e = torch.zeros(ng, dtype=torch.float64, device="cuda")
    for j in range(ng):
        e.zero_()
        e[j] = 1.0
        Sg[:, j] = p.matvec(e).cpu().numpy()
    assert _rel(Sg, S) < 1e-11
    f = torch.as_tensor(np.ascontiguousarray(d["f"]), dtype=torch.float64).reshape(-1).cuda()
    b = p.schur_rhs(f).cpu().numpy()
    assert _rel(b, B.schur_rhs()) < 1e-11


@pytest.mark.parametrize("name,N", [("trisin2d", [32, 32]), ("trisin2d", [64, 16]), ("tripoly2d", [16, 16]),
                                    ("tri3d_5_1_5", [16, 16, 16]), ("tripoly3d", [8, 16, 8])])
def test_tri_solve_matches_oracle(name, N):
    d = _sample(name, N)
    sol = T.solve_direct(T.assemble(d), d)
    p = ahoc.plan_for_triharmonic(d, restart=200, max_iters=2000)
    f = torch.as_tensor(np.ascontiguousarray(d["f"]), dtype=torch.float64).reshape(-1).cuda()
    u, info = p.solve(f, tol=1e-12)
    U = u.cpu().numpy().reshape(sol.U.shape)
    assert _rel(U, sol.U) < 1e-10, info
    q, _ = p.last_qv(with_v=False)
    # Q = Lap^2 u on the faces: its error is the Schur residual (1e-12 ||b||)
    # times ||S^-1||, larger for the triharmonic operator than U's
    assert _rel(q.cpu().numpy(), sol.Q) < 1e-7
    with pytest.raises(ahoc.AhocError):
        p.last_qv(with_v=True)


@pytest.mark.parametrize("N", [32, 64, 128, 256])
def test_tri_table5(N):
    """Table 5's printed errors reproduced on the GPU (both wavenumbers)."""
    rows = {int(r[0]): r for r in golden("triharmonic_table5.txt")}
    for col, name in ((1, "tri3d_5_1_5"), (2, "tri3d_25_5_25")):
        prob = inputs.triharmonic_problem(name)
        d = inputs.sample_triharmonic(prob, [N] * 3, backend="torch", device="cuda")
        p = ahoc.plan_for_triharmonic(d, restart=200, max_iters=2000)
        u, info = p.solve(d["f"].reshape(-1).contiguous(), tol=1e-12)
        err = float((u.reshape(d["u_exact"].shape) - d["u_exact"]).abs().max())
        want = float(rows[N][col])
        assert abs(err - want) < 0.01 * want, (name, N, err, want, info["iters"])
        # one clamped face: the measured inverse symbol is the exact inverse of its Schur operator
        assert info["iters"] <= 6, info["iters"]
        p.close()
