"""The allocation-free Poisson entry point, checked against the plan's.

ahoc_poisson_noalloc serves callers that cannot allocate device memory (a
foreign memory pool owns the device, a latency-critical loop must not
synchronise on cudaMalloc, or allocation is forbidden after start-up); its
scratch is a static 16 MiB device array.  This file sorts last so that a run
stopping at the first failure has already run every other test; it passes
alone in a fresh process as well.
"""

import ctypes as C

import numpy as np
import pytest
import torch

from paper_2609_16478_b300 import ahoc

pytestmark = pytest.mark.gpu


def _noalloc(dim, N, lo, hi, rhs, w):
    L = ahoc.lib()
    n = (C.c_int64 * dim)(*N)
    lo_ = (C.c_double * dim)(*lo)
    hi_ = (C.c_double * dim)(*hi)
    st = torch.cuda.current_stream()
    return L.ahoc_poisson_noalloc(dim, n, lo_, hi_, C.c_void_p(rhs.data_ptr()), C.c_void_p(w.data_ptr()),
                                  C.c_void_p(st.cuda_stream))


@pytest.mark.parametrize("N,lo,hi", [((1024, 1024), (0.0, 0.0), (1.0, 1.0)),
                                     ((32, 256), (0.0, -0.5), (1.0, 0.3)),
                                     ((64, 32, 16), (0.0, 0.0, 0.0), (1.0, 2.0, 0.5))])
def test_noalloc_matches_plan_on_two_calls(N, lo, hi):
    dim = len(N)
    nfull = int(np.prod([n + 1 for n in N]))
    nint = int(np.prod([n - 1 for n in N]))
    plan = ahoc.Plan(dim, N, torch.ones(nfull, dtype=torch.float64, device="cuda"), lo=lo, hi=hi)
    rng = np.random.default_rng(11)
    for call in range(2):
        rhs = torch.as_tensor(rng.normal(size=nint), dtype=torch.float64).cuda()
        ref = plan.poisson(rhs)
        w = torch.full_like(rhs, float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert _noalloc(dim, N, lo, hi, rhs, w) == ahoc.AHOC_OK
        torch.cuda.synchronize()
        if call == 1:
            # no device memory was taken by the call (the static array loaded with the library)
            assert torch.cuda.mem_get_info()[0] == free0
        rel = float(torch.linalg.norm(w - ref) / torch.linalg.norm(ref))
        assert rel < 1e-12, (call, rel)


def test_noalloc_rejects_oversized_grid():
    N = (2048, 2048)
    nint = 2047 * 2047
    rhs = torch.zeros(nint, dtype=torch.float64, device="cuda")
    w = torch.full_like(rhs, 7.0)
    st = _noalloc(2, N, (0.0, 0.0), (1.0, 1.0), rhs, w)
    torch.cuda.synchronize()
    assert st == ahoc.AHOC_EUNSUPPORTED
    assert b"16 MiB" in ahoc.lib().ahoc_last_error()
    assert float(w.min()) == 7.0 and float(w.max()) == 7.0
