"""Autotuner for launch shapes and serving batch sizes.

For a grid shape (dim, N) and a precision it measures, on the device, whole
solves of a seeded request of that shape (``inputs.sample_request``):

  * the chunk length of the tridiagonal solve along the last axis
    (``AHOC_TUNE_TRI_CHUNK``: 8, 16, 32 rows per thread);
  * the CTA size of the line DSTs (``AHOC_TUNE_DST_THREADS``: 128, 256, 512,
    1024 threads: the lines a CTA holds, hence the width of the row segments
    the y-transform reads and writes);
  * the FFT radix of the line DSTs (``AHOC_TUNE_DST_RADIX``: radix-4 or
    radix-8 stages: fewer passes over shared memory against more registers
    and half the threads busy in a radix-8 stage);
  * the batch size B of the serving plans: the per-problem time of a batched
    solve for B = 1, 2, 4, ... up to a memory cap; among the batches that
    finish within ``latency_factor`` times a single solve, the smallest B
    whose per-problem time is within ``slack`` of the best one (a larger
    batch only adds latency once the device is full).

Each choice is written to a JSON cache keyed "dim:N:prec" and applied to
the library's tuning table with ``apply``; ``batch_for`` turns a cache into
the server's per-shape batch function.  The selection rules are plain host
functions (``pick_fastest``, ``pick_batch``), testable without a GPU.
"""

from __future__ import annotations

import json
import os
import time
from typing import Callable, Dict, Iterable, List, Optional, Sequence, Tuple

TRI_CHOICES = (8, 16, 32)
CTA_CHOICES = (128, 256, 512, 1024)
RADIX_CHOICES = (4, 8)

# choices measured on a B300 for the serving shapes, mixed precision
# (``tune([(2, 128), ..., (3, 256)], "mixed", path=...)``); re-run to refresh
SHIPPED_MIXED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_b300_mixed.json")


def key(dim: int, N: int, prec: str) -> str:
    return "%d:%d:%s" % (dim, N, prec)


def pick_fastest(times: Dict[int, float]) -> int:
    """The candidate with the lowest time (ties: the first listed)."""
    best = min(times.values())
    return next(k for k, v in times.items() if v == best)


def pick_batch(per_problem_ms: Dict[int, float], slack: float = 0.05, latency_factor: float = 2.0) -> int:
    """Among the batches whose whole solve (B x per-problem time) takes at
    most latency_factor times a single solve, the smallest whose per-problem
    time is within slack of their best."""
    per = {int(b): t for b, t in per_problem_ms.items()}
    t1 = per.get(1, min(per.values()))
    ok = {b: t for b, t in per.items() if b * t <= latency_factor * t1 or b == 1}
    best = min(ok.values())
    return min(b for b, t in ok.items() if t <= best * (1 + slack))


def load(path: str) -> Dict[str, dict]:
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        return json.load(fh)


def save(path: str, cache: Dict[str, dict]) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(cache: Dict[str, dict]) -> None:
    """Write every cached launch shape into the library's tuning table."""
    from . import ahoc
    L = ahoc.lib()
    for k, v in cache.items():
        dim, N, prec = k.split(":")
        p = ahoc._prec(prec)
        if "tri_chunk" in v:
            ahoc._check(L.ahoc_tune_set(ahoc.AHOC_TUNE_TRI_CHUNK, int(dim), int(N), p, int(v["tri_chunk"])),
                        "ahoc_tune_set")
        if "dst_threads" in v:
            ahoc._check(L.ahoc_tune_set(ahoc.AHOC_TUNE_DST_THREADS, int(dim), int(N), p, int(v["dst_threads"])),
                        "ahoc_tune_set")
        if "dst_radix" in v:
            ahoc._check(L.ahoc_tune_set(ahoc.AHOC_TUNE_DST_RADIX, int(dim), int(N), p, int(v["dst_radix"])),
                        "ahoc_tune_set")


def batch_for(cache: Dict[str, dict], prec: str, default: Callable[[Tuple[int, int]], int]):
    """The server's per-shape batch function: the cached choice, else the default."""
    def f(k: Tuple[int, int]) -> int:
        v = cache.get(key(k[0], k[1], prec))
        return int(v["batch"]) if v and "batch" in v else default(k)
    return f


def _time_solves(dim, N, prec, B, reps=3, restart=60):
    import torch

    from . import ahoc, inputs
    specs = [inputs.RequestSpec(900 + r, dim, N, (r % 5,) * dim, 0.0) for r in range(B)]
    ds = [inputs.sample_request(s, device="cuda") for s in specs]
    alpha = torch.cat([d["alpha"] for d in ds])
    f = torch.cat([d["f"] for d in ds])
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        p = ahoc.Plan(dim, [N] * dim, alpha, prec=prec, batch=B, stream=st, restart=restart, max_iters=2000)
        u = torch.empty_like(f)
        p.solve(f, u, tol=1e-12, check=False)  # warm: graphs captured, caches filled
        st.synchronize()
        best = float("inf")
        for _ in range(reps):
            t0 = time.perf_counter()
            p.solve(f, u, tol=1e-12, check=False)
            st.synchronize()
            best = min(best, time.perf_counter() - t0)
        p.close()
    return best * 1e3


def tune_shape(dim: int, N: int, prec: str, batches: Sequence[int] = (1, 2, 4, 8, 16),
               mem_cap: float = 0.25, slack: float = 0.05, reps: int = 3, latency_factor: float = 2.0) -> dict:
    """Measure the four choices for one shape; the tuning table is left set."""
    import torch

    from . import ahoc
    L = ahoc.lib()
    p = ahoc._prec(prec)
    out: dict = {}
    # chunk length, with the built-in CTA and radix
    L.ahoc_tune_set(ahoc.AHOC_TUNE_DST_THREADS, dim, N, p, 0)
    L.ahoc_tune_set(ahoc.AHOC_TUNE_DST_RADIX, dim, N, p, 0)
    tri = {}
    for c in TRI_CHOICES:
        ahoc._check(L.ahoc_tune_set(ahoc.AHOC_TUNE_TRI_CHUNK, dim, N, p, c), "ahoc_tune_set")
        tri[c] = _time_solves(dim, N, prec, 1, reps)
    out["tri_chunk"] = pick_fastest(tri)
    ahoc._check(L.ahoc_tune_set(ahoc.AHOC_TUNE_TRI_CHUNK, dim, N, p, out["tri_chunk"]), "ahoc_tune_set")
    # CTA size of the line DSTs (only differs when 512 threads hold more than one line)
    cta = {}
    for c in CTA_CHOICES if N // 8 < 512 else (512,):
        ahoc._check(L.ahoc_tune_set(ahoc.AHOC_TUNE_DST_THREADS, dim, N, p, c), "ahoc_tune_set")
        cta[c] = _time_solves(dim, N, prec, 1, reps)
    out["dst_threads"] = pick_fastest(cta)
    ahoc._check(L.ahoc_tune_set(ahoc.AHOC_TUNE_DST_THREADS, dim, N, p, out["dst_threads"]), "ahoc_tune_set")
    # FFT radix, with the chosen CTA
    rad = {}
    for r in RADIX_CHOICES:
        ahoc._check(L.ahoc_tune_set(ahoc.AHOC_TUNE_DST_RADIX, dim, N, p, r), "ahoc_tune_set")
        rad[r] = _time_solves(dim, N, prec, 1, reps)
    out["dst_radix"] = pick_fastest(rad)
    ahoc._check(L.ahoc_tune_set(ahoc.AHOC_TUNE_DST_RADIX, dim, N, p, out["dst_radix"]), "ahoc_tune_set")
    # batch size under a device-memory cap
    free, _ = torch.cuda.mem_get_info()
    per = {}
    for B in batches:
        need = ahoc.workspace_bytes(dim, [N] * dim, 60, prec, -1, B) + 4 * B * (N + 1) ** dim * 8
        if need > mem_cap * free:
            break
        per[B] = _time_solves(dim, N, prec, B, reps) / B
    out["batch"] = pick_batch(per, slack, latency_factor)
    out["ms"] = {"tri_chunk": tri, "dst_threads": cta, "dst_radix": rad, "per_problem_by_batch": per}
    return out


def tune(shapes: Iterable[Tuple[int, int]], prec: str, path: Optional[str] = None, **kw) -> Dict[str, dict]:
    """Tune every (dim, N) not yet in the cache at `path`; save and apply."""
    cache = load(path) if path else {}
    for dim, N in shapes:
        k = key(dim, N, prec)
        if k not in cache:
            cache[k] = tune_shape(dim, N, prec, **kw)
            if path:
                save(path, cache)
    apply(cache)
    return cache
