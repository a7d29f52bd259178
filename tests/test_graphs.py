"""GMRES iterations replayed as CUDA graphs give the bits of plain launches."""

import pytest
import torch

from paper_2609_16478_b300 import ahoc, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,N,prec,B", [(2, 64, "fp64", 1), (2, 256, "fp64", 3), (2, 128, "mixed", 2),
                                          (3, 32, "fp64", 2), (3, 32, "mixed", 1)])
def test_graphs_equal_plain(dim, N, prec, B):
    specs = [inputs.RequestSpec(20 + r, dim, N, (r % 5,) * dim, 0.0) for r in range(B)]
    ds = [inputs.sample_request(s, device="cuda") for s in specs]
    alpha = torch.cat([d["alpha"] for d in ds])
    f = torch.cat([d["f"] for d in ds])
    out = {}
    for graphs in (False, True):
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            p = ahoc.Plan(dim, [N] * dim, alpha, prec=prec, batch=B, stream=st, graphs=graphs, restart=40)
            u1, i1 = p.solve(f, tol=1e-12)
            u2, i2 = p.solve(f, tol=1e-12)  # the second solve replays the captured graphs
        st.synchronize()
        i1 = i1 if B > 1 else [i1]
        i2 = i2 if B > 1 else [i2]
        assert torch.equal(u1, u2)
        assert [x["iters"] for x in i1] == [x["iters"] for x in i2]
        assert i1[0]["launches"] == i2[0]["launches"]
        out[graphs] = (u2, i2)
        p.close()
    assert torch.equal(out[False][0], out[True][0])
    assert [x["iters"] for x in out[False][1]] == [x["iters"] for x in out[True][1]]
    assert out[False][1][0]["launches"] == out[True][1][0]["launches"]
