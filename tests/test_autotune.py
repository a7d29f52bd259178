"""Autotuner: selection rules and cache on the host; the library's tuning
table through the C ABI (no device work); tuned shapes on the GPU."""

import os

import pytest

from paper_2609_16478_b300 import ahoc, autotune


def test_pick_rules():
    assert autotune.pick_fastest({8: 3.0, 16: 2.0, 32: 2.5}) == 16
    assert autotune.pick_fastest({128: 1.0, 256: 1.0}) == 128
    # per-problem times fall, then flatten: the smallest batch within 5% of the best
    assert autotune.pick_batch({1: 10.0, 2: 5.5, 4: 3.1, 8: 3.0, 16: 3.05}, latency_factor=100) == 4
    assert autotune.pick_batch({1: 2.0, 2: 2.5}) == 1
    # ... among the batches that finish within twice a single solve (B * t_B <= 2 t_1)
    assert autotune.pick_batch({1: 10.0, 2: 5.5, 4: 3.1, 8: 3.0, 16: 3.05}) == 4  # 12.4 <= 20 < 24
    assert autotune.pick_batch({1: 81.3, 2: 75.0, 4: 70.8, 8: 69.4}) == 2
    assert autotune.pick_batch({"1": 4.3, "2": 2.35, "16": 0.36}) == 16


def test_cache_roundtrip_and_batch_for(tmp_path):
    path = os.path.join(tmp_path, "tune.json")
    cache = {autotune.key(2, 128, "mixed"): {"tri_chunk": 16, "dst_threads": 256, "batch": 8}}
    autotune.save(path, cache)
    assert autotune.load(path) == cache
    f = autotune.batch_for(cache, "mixed", lambda k: 1)
    assert f((2, 128)) == 8 and f((3, 64)) == 1


def test_tuning_table_through_abi():
    L = ahoc.lib()
    k, dim, N, prec = ahoc.AHOC_TUNE_TRI_CHUNK, 2, 512, ahoc.AHOC_MIXED
    assert L.ahoc_tune_get(k, dim, N, prec) == 0
    assert L.ahoc_tune_set(k, dim, N, prec, 8) == ahoc.AHOC_OK
    assert L.ahoc_tune_get(k, dim, N, prec) == 8
    assert L.ahoc_tune_set(k, dim, N, prec, 12) == ahoc.AHOC_EINVAL  # not offered
    assert L.ahoc_tune_set(ahoc.AHOC_TUNE_DST_THREADS, dim, N, prec, 2048) == ahoc.AHOC_EINVAL
    for r, want in ((4, ahoc.AHOC_OK), (8, ahoc.AHOC_OK), (2, ahoc.AHOC_EINVAL), (16, ahoc.AHOC_EINVAL)):
        assert L.ahoc_tune_set(ahoc.AHOC_TUNE_DST_RADIX, dim, N, prec, r) == want
    assert L.ahoc_tune_get(ahoc.AHOC_TUNE_DST_RADIX, dim, N, prec) == 8
    assert L.ahoc_tune_set(ahoc.AHOC_TUNE_DST_RADIX, dim, N, prec, 0) == ahoc.AHOC_OK
    assert L.ahoc_tune_set(k, 4, N, prec, 8) == ahoc.AHOC_EINVAL
    assert L.ahoc_tune_get(k, dim, 500, prec) == -1
    # the chunk length sets the tridiagonal scratch, so the workspace follows the table
    b8 = ahoc.workspace_bytes(2, [512, 512], 60, "mixed")
    assert L.ahoc_tune_set(k, dim, N, prec, 32) == ahoc.AHOC_OK
    b32 = ahoc.workspace_bytes(2, [512, 512], 60, "mixed")
    assert b8 > b32
    assert L.ahoc_tune_set(k, dim, N, prec, 0) == ahoc.AHOC_OK


@pytest.mark.gpu
@pytest.mark.parametrize("dim,N,prec", [(2, 128, "mixed"), (3, 16, "fp64"), (3, 16, "mixed")])
def test_tuned_shapes_same_solution(dim, N, prec):
    """Every offered shape solves the same discrete problem: each result
    against the CPU oracle's direct solve of the request, and the tuner
    returns a complete entry."""
    import numpy as np
    import torch

    from oracle import coupled
    from paper_2609_16478_b300 import inputs
    spec = inputs.RequestSpec(5, dim, N, (2,) * dim, 0.0)
    d = inputs.sample_request(spec, device="cuda")
    h = inputs.request_numpy(spec)
    ref = coupled.solve_direct(coupled.assemble(h), h).U
    L = ahoc.lib()
    p_ = ahoc._prec(prec)
    for tri in autotune.TRI_CHOICES:
        for cta in autotune.CTA_CHOICES:
            for rad in autotune.RADIX_CHOICES:
                L.ahoc_tune_set(ahoc.AHOC_TUNE_TRI_CHUNK, dim, N, p_, tri)
                L.ahoc_tune_set(ahoc.AHOC_TUNE_DST_THREADS, dim, N, p_, cta)
                L.ahoc_tune_set(ahoc.AHOC_TUNE_DST_RADIX, dim, N, p_, rad)
                p = ahoc.Plan(dim, [N] * dim, d["alpha"], prec=prec)
                u, info = p.solve(d["f"], tol=1e-12)
                U = u.cpu().numpy().reshape(ref.shape)
                rel = np.linalg.norm(U - ref) / np.linalg.norm(ref)
                assert rel < (1e-10 if prec == "fp64" else 1e-9), (tri, cta, rad, rel)
                p.close()
    entry = autotune.tune_shape(dim, N, prec, batches=(1, 2, 4), reps=1)
    assert entry["tri_chunk"] in autotune.TRI_CHOICES and entry["dst_threads"] in autotune.CTA_CHOICES
    assert entry["dst_radix"] in autotune.RADIX_CHOICES and entry["batch"] in (1, 2, 4)
    for k in (ahoc.AHOC_TUNE_TRI_CHUNK, ahoc.AHOC_TUNE_DST_THREADS, ahoc.AHOC_TUNE_DST_RADIX):
        L.ahoc_tune_set(k, dim, N, p_, 0)
