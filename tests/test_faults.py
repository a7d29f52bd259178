"""Failure handling, made on the host (no GPU fault): a NaN in one problem's
data, an iteration cap, and a bad request inside a served batch.

A problem whose data or iterates turn NaN or Inf is masked out of its batch
like a converged one: it reports AHOC_ENUMERIC and the other problems get
the bits of their own solves.  A solve that hits max_iters reports
AHOC_ENOCONV with the best iterate in u.
"""


import numpy as np
import pytest
import torch

from paper_2609_16478_b300 import ahoc, inputs, serving

pytestmark = pytest.mark.gpu


def _reqs(dim, N, B):
    specs = [inputs.RequestSpec(r, dim, N, ((r % 3),) * dim, 0.0) for r in range(B)]
    return specs, [inputs.sample_request(s, device="cuda") for s in specs]


@pytest.mark.parametrize("dim,N,prec,where", [(2, 64, "fp64", "f"), (2, 64, "mixed", "f"), (3, 16, "fp64", "f"),
                                              (2, 64, "fp64", "alpha"), (3, 16, "mixed", "alpha")])
def test_nan_problem_masked_out_of_its_batch(dim, N, prec, where):
    B = 3
    _, ds = _reqs(dim, N, B)
    nf = (N + 1) ** dim
    alpha = torch.cat([d["alpha"] for d in ds])
    f = torch.cat([d["f"] for d in ds])
    bad = 1
    if where == "f":
        f[bad * nf + nf // 2] = float("nan")
    else:
        # a NaN in alpha at a face point (2D: (1, 0); 3D: (1, 1, 0)) reaches the traces
        alpha[bad * nf + (1 if dim == 2 else N + 2)] = float("nan")
    pb = ahoc.Plan(dim, [N] * dim, alpha, prec=prec, batch=B)
    u, infos = pb.solve(f, tol=1e-12, check=False)
    assert infos[bad]["status"] == ahoc.AHOC_ENUMERIC, infos[bad]
    for b in (0, 2):
        assert infos[b]["status"] == 0
        ps = ahoc.Plan(dim, [N] * dim, ds[b]["alpha"], prec=prec)
        us, info = ps.solve(ds[b]["f"], tol=1e-12)
        assert torch.equal(u[b * nf:(b + 1) * nf], us), b
        assert infos[b]["iters"] == info["iters"]
    with pytest.raises(ahoc.AhocError) as e:
        pb.solve(f, tol=1e-12)
    assert e.value.status == ahoc.AHOC_ENUMERIC


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_max_iters_cap_returns_best_iterate(prec):
    """ENOCONV with u from the last iterate: its Schur residual is the one
    GMRES reports, and more iterations give a better u."""
    specs, ds = _reqs(2, 128, 1)
    d = ds[0]
    u_ref, _ = ahoc.Plan(2, [128, 128], d["alpha"], prec=prec, levels=0).solve(d["f"], tol=1e-12)
    errs = []
    for cap in (3, 6):
        p = ahoc.Plan(2, [128, 128], d["alpha"], prec=prec, levels=0, max_iters=cap)
        u, info = p.solve(d["f"], tol=1e-12, check=False)
        assert info["status"] == ahoc.AHOC_ENOCONV and info["iters"] == cap, info
        assert torch.isfinite(u).all()
        errs.append(float(torch.linalg.norm(u - u_ref) / torch.linalg.norm(u_ref)))
    assert errs[1] < errs[0] < 1.0, errs


def test_server_isolates_a_bad_request():
    specs = inputs.request_stream(8, rate=0.0, seed=3, p2d=1.0, sizes2d=(64,))
    bad = specs[2].rid

    def poison(spec, alpha, f):
        if spec.rid == bad:
            f[len(f) // 2] = float("nan")

    srv = serving.Server(prec="mixed", tol=1e-12, workers=2, keep_results=True, batch_for=lambda k: 4)
    srv.data_hook = poison
    recs = srv.run(specs, realtime=False)
    srv.close()
    by = {r.rid: r for r in recs}
    assert by[bad].status == ahoc.AHOC_ENUMERIC
    assert max(r.batch for r in recs) > 1
    for s in specs:
        if s.rid == bad:
            continue
        d = inputs.sample_request(s, device="cuda")
        u, _ = ahoc.Plan(2, [64, 64], d["alpha"], prec="mixed", restart=srv.restart, max_iters=2000).solve(
            d["f"], tol=1e-12)
        assert by[s.rid].status == 0 and torch.equal(srv.results[s.rid], u)


def test_server_deadline_and_cancel():
    specs = inputs.request_stream(12, rate=0.0, seed=4, p2d=1.0, sizes2d=(128,))
    specs[5].deadline = -1.0  # already expired when it is first considered
    srv = serving.Server(prec="mixed", tol=1e-10, workers=1, batch_for=lambda k: 2)
    # two requests are withdrawn right after they arrive, before a worker can take them
    orig_arrive = srv.sched.arrive
    cancelled = []

    def arrive(req):
        orig_arrive(req)
        if req.rid in (9, 10):
            cancelled.append(srv.cancel(req.rid))

    srv.sched.arrive = arrive
    recs = srv.run(specs, realtime=False)
    srv.close()
    by = {r.rid: r for r in recs}
    assert by[specs[5].rid].status == serving.STATUS_EXPIRED
    assert cancelled == [True, True]
    assert by[9].status == by[10].status == serving.STATUS_CANCELLED
    done = [r for r in recs if r.status == 0]
    assert len(done) == 12 - 3
    s = serving.summarize(recs)
    assert s["dropped"] == 3 and s["requests"] == 9
