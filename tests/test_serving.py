"""The request server: each result is the same alone and in the mix.

Requests of several shapes are served by concurrent batched plans; every
result must equal (bit for bit) the solve of the same request on a
single-problem plan with the same settings, and must reach the stated
accuracy against the exact solution.
"""

import pytest
import torch

from paper_2609_16478_b300 import ahoc, inputs, serving

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,realtime", [("mixed", False), ("fp64", True)])
def test_served_equals_solo(prec, realtime):
    specs = inputs.request_stream(20, rate=400.0 if realtime else 0.0, seed=9, sizes2d=(64, 128), sizes3d=(16, 32))
    srv = serving.Server(prec=prec, tol=1e-10, workers=3, keep_results=True, batch_for=lambda k: 4,
                         check_exact=True)
    recs = srv.run(specs, realtime=realtime)
    srv.close()
    assert all(r.status == 0 for r in recs)
    assert max(r.batch for r in recs) > 1  # requests were batched
    for spec, rec in zip(specs, recs):
        d = inputs.sample_request(spec, device="cuda", with_exact=True)
        p = ahoc.Plan(spec.dim, [spec.N] * spec.dim, d["alpha"], prec=prec, restart=srv.restart, max_iters=2000)
        u, info = p.solve(d["f"], tol=1e-10)
        assert torch.equal(srv.results[spec.rid], u), spec
        assert info["iters"] == rec.iters
        # discretisation-level error against the exact solution
        assert rec.err_inf == float((u - d["u_exact"]).abs().max())
        assert rec.err_inf < 5e-3
        p.close()
    s = serving.summarize(recs)
    assert s["p99_ms"] >= s["p50_ms"] > 0 and s["dof_per_s"] > 0
