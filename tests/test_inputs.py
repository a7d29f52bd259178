"""The serving request generator's closed-form data against the symbolic path."""

import numpy as np
import pytest
import sympy as sp

from paper_2609_16478_b300 import inputs


@pytest.mark.parametrize("spec", [inputs.RequestSpec(7, 2, 16, (3, 1), 0.0),
                                  inputs.RequestSpec(11, 3, 8, (0, 4, 2), 0.0)])
def test_request_matches_symbolic(spec):
    d = inputs.sample_request(spec, device="cpu", with_exact=True)
    x = inputs.X[:spec.dim]
    u = 1
    for a in range(spec.dim):
        u = u * sp.sin(sp.pi * x[a]) ** 2 * sp.cos(spec.m[a] * sp.pi * x[a])
    ref = inputs.sample(inputs.Problem("t", spec.dim, inputs.fourier_alpha(spec.dim, 6, 4, 0.5, spec.rid), u),
                        [spec.N] * spec.dim)
    for k in ("alpha", "f", "u_exact"):
        a = d[k].numpy().reshape(ref[k].shape)
        assert np.max(np.abs(a - ref[k])) <= 1e-13 * np.max(np.abs(ref[k])), k
    # the request data are all zero on the boundary: g_D, g_N, tangential Laplacian, edge v
    for k in ("g_D", "g_N", "lapt_gD", "v_edge"):
        assert np.max(np.abs(ref[k])) < 1e-12, k


def test_request_stream_mix():
    s = inputs.request_stream(2000, 50.0, seed=5)
    assert [r.rid for r in s] == list(range(2000))
    t = np.array([r.arrival for r in s])
    assert np.all(np.diff(t) > 0)
    assert abs(t[-1] / 2000 - 1 / 50.0) < 0.1 / 50.0  # mean gap close to 1/rate
    frac2d = np.mean([r.dim == 2 for r in s])
    assert 0.66 < frac2d < 0.74
    assert {r.N for r in s if r.dim == 2} == set(inputs.SERVE_2D)
    assert {r.N for r in s if r.dim == 3} == set(inputs.SERVE_3D)
    assert all(0 <= v <= 4 for r in s for v in r.m)
    assert s[17] == inputs.request_stream(2000, 50.0, seed=5)[17]  # reproducible


@pytest.mark.parametrize("dim,M,K,A,seed", [(2, 8, 6, 0.4, 1), (3, 6, 4, 0.4, 2), (3, 6, 4, 0.5, 3)])
def test_fourier_coefficient_recipe(dim, M, K, A, seed):
    """The seeded coefficient fields of the Fourier-coefficient workloads:
    modes drawn with 0 <= k_a <= K and k != 0, alpha = 1 + A phi / max|phi|
    with the maximum taken on a fixed lattice (1024 points per axis in 2D,
    128 in 3D), so alpha reaches 1 +- A there, stays positive everywhere,
    does not depend on the solve's grid, and is the same for the same seed."""
    modes = inputs.fourier_modes(dim, M, K, seed)
    assert len(modes) == M
    assert all(any(k) and all(0 <= v <= K for v in k) for k, _, _ in modes)
    assert all(-1 <= c <= 1 and 0 <= th <= 2 * np.pi for _, c, th in modes)
    assert modes == inputs.fourier_modes(dim, M, K, seed)
    alpha = sp.lambdify(inputs.X[:dim], inputs.fourier_alpha(dim, M, K, A, seed), "numpy")
    L = 1024 if dim == 2 else 128
    t = np.linspace(0.0, 1.0, L + 1)
    lat = alpha(*np.meshgrid(*([t] * dim), indexing="ij"))
    assert abs(np.max(np.abs(lat - 1)) - A) < 1e-12
    pts = np.random.default_rng(0).uniform(size=(dim, 20000))
    vals = alpha(*pts)
    # between lattice points |phi| may exceed its lattice maximum by the
    # lattice's second-order error only
    assert np.max(np.abs(vals - 1)) < A * (1 + 2e-3)
    assert np.min(vals) > 0
