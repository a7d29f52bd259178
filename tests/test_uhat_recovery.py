"""Recovery of U from the U-hat slots (2D FP64, constant beta/alpha).

U is linear in Q, so the U-hat fields that the Schur matvecs of GMRES's first
cycle leave behind, combined with the GMRES coefficients and transformed back
once, give the U of the two recovery Poisson solves (Algorithm 1) up to
rounding.  The slots are compared with the plain recovery (uhat_slots=-1) on
the same inputs: u, Q and V from ahoc_last_qv; the fallbacks (a restart,
more steps than slots) take the plain recovery and give its bits.
"""

import pytest
import torch

from paper_2609_16478_b300 import ahoc, inputs

pytestmark = pytest.mark.gpu


def _solve(data, N, **kw):
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        p = ahoc.plan_for(data, device="cuda", stream=st, **kw)
        f = data["f"].reshape(-1).contiguous()
        u, info = p.solve(f, tol=1e-12)
        q, v = p.last_qv()
        st.synchronize()
        p.close()
    return u, q, v, info


@pytest.mark.parametrize("name,N,levels", [("fourier2d", 256, -1), ("fourier2d", 512, 0), ("navier2d", 256, -1),
                                           ("shift2d", 256, 0)])
def test_slots_match_two_solves(name, N, levels):
    prob = inputs.config_problem(name)
    data = inputs.sample(prob, [N, N], backend="torch", device="cuda")
    ua, qa, va, ia = _solve(data, N, levels=levels, restart=100, uhat_slots=64)
    ub, qb, vb, ib = _solve(data, N, levels=levels, restart=100, uhat_slots=-1)
    assert ia["iters"] == ib["iters"] and ia["iters"] <= 64
    # the slot path replaces four DSTs of the recovery by one
    assert ib["kernel_launches"]["dst_x"] - ia["kernel_launches"]["dst_x"] == 3
    assert torch.equal(qa, qb)
    scale = float(ub.abs().max())
    assert float((ua - ub).abs().max()) <= 1e-12 * scale
    assert float((va - vb).abs().max()) <= 1e-12 * float(vb.abs().max())
    err_a = float((ua.reshape(N + 1, N + 1) - data["u_exact"]).abs().max())
    err_b = float((ub.reshape(N + 1, N + 1) - data["u_exact"]).abs().max())
    assert abs(err_a / err_b - 1) < 1e-3


@pytest.mark.parametrize("kw", [dict(restart=3, levels=0), dict(uhat_slots=2, levels=0)])
def test_fallback_gives_plain_bits(kw):
    N = 128
    data = inputs.sample(inputs.config_problem("fourier2d"), [N, N], backend="torch", device="cuda")
    ua, qa, va, ia = _solve(data, N, **kw)
    kb = dict(kw)
    kb["uhat_slots"] = -1
    ub, qb, vb, ib = _solve(data, N, **kb)
    assert ia["iters"] > 3
    assert torch.equal(ua, ub) and torch.equal(qa, qb) and torch.equal(va, vb)


def test_batch_slots_match_solo():
    N, B = 128, 3
    specs = [inputs.RequestSpec(40 + r, 2, N, (r,) * 2, 0.0) for r in range(B)]
    ds = [inputs.sample_request(s, device="cuda") for s in specs]
    alpha = torch.cat([d["alpha"] for d in ds])
    f = torch.cat([d["f"] for d in ds])
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        p = ahoc.Plan(2, [N, N], alpha, batch=B, stream=st, restart=60)
        u, infos = p.solve(f, tol=1e-12)
        p.close()
        solo = []
        for d in ds:
            ps = ahoc.Plan(2, [N, N], d["alpha"], stream=st, restart=60, uhat_slots=-1)
            us, _ = ps.solve(d["f"], tol=1e-12)
            solo.append(us)
            ps.close()
    st.synchronize()
    nf = (N + 1) ** 2
    for b in range(B):
        ub = u[b * nf:(b + 1) * nf]
        assert float((ub - solo[b]).abs().max()) <= 1e-12 * float(solo[b].abs().max())
