"""The request server: each result is the same alone and in the mix.

Requests of several shapes are served by concurrent batched plans; every
result must equal (bit for bit) the solve of the same request on a
single-problem plan with the same settings, match the CPU oracle's direct
solve of that request (where the oracle is quick: 2D, and 3D at N = 16), and
reach the oracle's (or the FP64 solve's) discretisation error to within 5%.
"""

import numpy as np
import pytest
import torch

from oracle import coupled
from paper_2609_16478_b300 import ahoc, inputs, serving

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,realtime", [("mixed", False), ("fp64", True)])
def test_served_equals_solo(prec, realtime):
    tol = 1e-12
    specs = inputs.request_stream(20, rate=400.0 if realtime else 0.0, seed=9, sizes2d=(64, 128), sizes3d=(16, 32))
    srv = serving.Server(prec=prec, tol=tol, workers=3, keep_results=True, batch_for=lambda k: 4,
                         check_exact=True)
    recs = srv.run(specs, realtime=realtime)
    srv.close()
    assert all(r.status == 0 for r in recs)
    if not realtime:
        # every request queued at once: same-shape requests meet in a batch.
        # (With arrivals in real time, batching depends on how fast the
        # feeder and the workers run; this case checks the results.)
        assert max(r.batch for r in recs) > 1
    n_oracle = 0
    for spec, rec in zip(specs, recs):
        d = inputs.sample_request(spec, device="cuda", with_exact=True)
        p = ahoc.Plan(spec.dim, [spec.N] * spec.dim, d["alpha"], prec=prec, restart=srv.restart, max_iters=2000)
        u, info = p.solve(d["f"], tol=tol)
        assert torch.equal(srv.results[spec.rid], u), spec
        assert info["iters"] == rec.iters
        assert rec.err_inf == float((u - d["u_exact"]).abs().max())
        p.close()
        if spec.dim == 2 or spec.N == 16:
            # the oracle's direct solve of the same request
            h = inputs.request_numpy(spec)
            sol = coupled.solve_direct(coupled.assemble(h), h)
            U = u.cpu().numpy().reshape(sol.U.shape)
            rel = np.linalg.norm(U - sol.U) / np.linalg.norm(sol.U)
            assert rel < (1e-10 if prec == "fp64" else 1e-9), (spec, rel)
            err_ref = float(np.max(np.abs(sol.U - h["u_exact"])))
            n_oracle += 1
        else:
            p64 = ahoc.Plan(spec.dim, [spec.N] * spec.dim, d["alpha"], restart=srv.restart, max_iters=2000)
            u64, _ = p64.solve(d["f"], tol=tol)
            err_ref = float((u64 - d["u_exact"]).abs().max())
            p64.close()
        # the served result reaches the discretisation error of the exact discrete solution
        assert rec.err_inf <= 1.05 * err_ref, (spec, rec.err_inf, err_ref)
    assert n_oracle >= 10
    s = serving.summarize(recs)
    assert s["p99_ms"] >= s["p50_ms"] > 0 and s["dof_per_s"] > 0
