"""Thin ctypes binding of the C ABI in ``include/ahoc.h`` (argument marshalling only).

Every array argument is a CUDA float64 tensor whose ``data_ptr()`` is passed
straight to the library; work runs on the plan's stream (by default torch's
current stream at plan creation).  Nothing here computes: there is no CPU or
PyTorch fallback, and :func:`lib` raises if the shared library is missing.
"""

from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libahoc.so")

AHOC_OK, AHOC_EINVAL, AHOC_ENOMEM, AHOC_ECUDA, AHOC_ENOCONV, AHOC_ENUMERIC, AHOC_ETIMEOUT, \
    AHOC_EUNSUPPORTED, AHOC_EINTERNAL = range(9)
AHOC_FP64, AHOC_MIXED = 0, 1
AHOC_TUNE_TRI_CHUNK, AHOC_TUNE_DST_THREADS, AHOC_TUNE_DST_RADIX = 0, 1, 2

# every entry point declared in include/ahoc.h
SYMBOLS = ("ahoc_workspace_bytes", "ahoc_plan_create", "ahoc_solve", "ahoc_solve_host", "ahoc_solve_from",
           "ahoc_matvec", "ahoc_schur_rhs", "ahoc_last_qv", "ahoc_dst1", "ahoc_poisson", "ahoc_plan_destroy", "ahoc_status_string",
           "ahoc_last_error", "ahoc_n_gamma", "ahoc_poisson_noalloc", "ahoc_plan_load", "ahoc_set_active",
           "ahoc_batch", "ahoc_tune_set", "ahoc_tune_get")


class ahoc_bdata(C.Structure):
    _fields_ = [("g_D", C.c_void_p), ("g_N", C.c_void_p), ("lapt_gD", C.c_void_p), ("v_edge", C.c_void_p),
                ("g_L", C.c_void_p), ("beta", C.c_void_p), ("lap_gD", C.c_void_p), ("bilap", C.c_void_p),
                ("g_NN", C.c_void_p), ("lapt_w", C.c_void_p)]


AHOC_NK = 8
KERNEL_NAMES = ("dst_x", "dst_y", "tri", "vrhs", "urhs", "trace", "krylov", "other")


class ahoc_opts(C.Structure):
    _fields_ = [("prec", C.c_int), ("max_iters", C.c_int), ("restart", C.c_int), ("precond", C.c_int),
                ("refine_tol", C.c_double), ("timing", C.c_int), ("workspace", C.c_void_p),
                ("workspace_bytes", C.c_size_t), ("levels", C.c_int), ("coarse_tol", C.c_double),
                ("batch", C.c_int), ("navier", C.c_int), ("shift", C.c_double), ("no_graphs", C.c_int),
                ("variable_beta", C.c_int), ("uhat_slots", C.c_int), ("unfused", C.c_int),
                ("triharmonic", C.c_int), ("auto_shift", C.c_int), ("first32", C.c_int)]


class ahoc_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("rel_resid", C.c_double),
                ("ms_total", C.c_double), ("ms_matvec", C.c_double), ("launches", C.c_int64),
                ("kernel_ms", C.c_double * AHOC_NK), ("kernel_launches", C.c_int64 * AHOC_NK),
                ("levels", C.c_int), ("coarse_iters", C.c_int),
                ("kernel_ms_top", C.c_double * AHOC_NK), ("kernel_launches_top", C.c_int64 * AHOC_NK),
                ("refine_steps", C.c_int), ("refine_hist", C.c_double * 16), ("inner_iters", C.c_int * 16),
                ("refine_du", C.c_double * 16), ("status", C.c_int), ("vsolve_iters", C.c_int)]


class AhocError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(what)
        self.status = status


_lib = None


def lib():
    """Load the in-tree ``libahoc.so`` (build it with ``python -m paper_2609_16478_b300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libahoc.so not built: run `python -m paper_2609_16478_b300.build` (no fallback exists)")
    L = C.CDLL(LIB_PATH)
    i64p = C.POINTER(C.c_int64)
    dp = C.POINTER(C.c_double)
    L.ahoc_workspace_bytes.argtypes = [C.c_int, i64p, C.POINTER(ahoc_opts), C.POINTER(C.c_size_t)]
    L.ahoc_plan_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, i64p, dp, dp, C.c_void_p,
                                   C.POINTER(ahoc_bdata), C.POINTER(ahoc_opts), C.c_void_p]
    L.ahoc_solve.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.POINTER(ahoc_info)]
    L.ahoc_solve_from.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.POINTER(ahoc_info)]
    L.ahoc_solve_host.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.POINTER(ahoc_info)]
    L.ahoc_matvec.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    L.ahoc_schur_rhs.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    L.ahoc_last_qv.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    L.ahoc_dst1.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_double]
    L.ahoc_poisson.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    L.ahoc_plan_destroy.argtypes = [C.c_void_p]
    L.ahoc_status_string.argtypes = [C.c_int]
    L.ahoc_status_string.restype = C.c_char_p
    L.ahoc_last_error.argtypes = []
    L.ahoc_last_error.restype = C.c_char_p
    L.ahoc_poisson_noalloc.argtypes = [C.c_int, i64p, dp, dp, C.c_void_p, C.c_void_p, C.c_void_p]
    L.ahoc_poisson_noalloc.restype = C.c_int
    L.ahoc_n_gamma.argtypes = [C.c_void_p]
    L.ahoc_n_gamma.restype = C.c_int64
    L.ahoc_plan_load.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(ahoc_bdata)]
    L.ahoc_set_active.argtypes = [C.c_void_p, C.POINTER(C.c_int)]
    L.ahoc_batch.argtypes = [C.c_void_p]
    L.ahoc_batch.restype = C.c_int
    L.ahoc_tune_set.argtypes = [C.c_int, C.c_int, C.c_int64, C.c_int, C.c_int]
    L.ahoc_tune_set.restype = C.c_int
    L.ahoc_tune_get.argtypes = [C.c_int, C.c_int, C.c_int64, C.c_int]
    L.ahoc_tune_get.restype = C.c_int
    for name in ("ahoc_workspace_bytes", "ahoc_plan_create", "ahoc_solve", "ahoc_solve_host", "ahoc_solve_from",
                 "ahoc_matvec", "ahoc_schur_rhs", "ahoc_last_qv", "ahoc_dst1", "ahoc_poisson", "ahoc_plan_destroy",
                 "ahoc_plan_load", "ahoc_set_active"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(status: int, call: str):
    if status != AHOC_OK:
        L = lib()
        raise AhocError(status, "%s: %s (%s)" % (call, L.ahoc_status_string(status).decode(),
                                                 L.ahoc_last_error().decode()))


def _ptr(t: Optional[torch.Tensor], numel: int, name: str):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("%s must be a contiguous CUDA float64 tensor" % name)
    if t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), numel))
    return C.c_void_p(t.data_ptr())


def _hptr(t: torch.Tensor, numel: int, name: str):
    if not (t.device.type == "cpu" and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("%s must be a contiguous host float64 tensor" % name)
    if t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), numel))
    return C.c_void_p(t.data_ptr())


def _prec(prec) -> int:
    """AHOC_FP64 / AHOC_MIXED from an int or "fp64" / "mixed"."""
    if isinstance(prec, str):
        return {"fp64": AHOC_FP64, "mixed": AHOC_MIXED}[prec]
    return int(prec)


def _opts(prec, max_iters, restart, precond, workspace=None, timing=0, levels=-1, refine_tol=0.0, coarse_tol=0.0,
          batch=1, graphs=True, navier=0, shift=0.0, variable_beta=False, uhat_slots=0, fused=True,
          triharmonic=False, auto_shift=False, first32=False):
    o = ahoc_opts()
    o.auto_shift = 1 if auto_shift else 0
    o.first32 = 1 if first32 else 0
    o.unfused = 0 if fused else 1
    o.triharmonic = 1 if triharmonic else 0
    o.variable_beta = 1 if variable_beta else 0
    o.uhat_slots = int(uhat_slots)
    o.batch = int(batch)
    o.navier = int(navier)
    o.shift = float(shift)
    o.no_graphs = 0 if graphs else 1
    o.coarse_tol = float(coarse_tol)
    o.timing = int(timing)
    o.levels = int(levels)
    o.prec = _prec(prec)
    o.max_iters = max_iters
    o.restart = restart
    o.precond = precond
    o.refine_tol = float(refine_tol)
    if workspace is not None:
        o.workspace = C.c_void_p(workspace.data_ptr())
        o.workspace_bytes = workspace.numel()
    return o


def workspace_bytes(dim: int, N: Sequence[int], restart: int = 100, prec: int = AHOC_FP64, levels: int = -1,
                    batch: int = 1, shift: float = 0.0, variable_beta: bool = False, uhat_slots: int = 0,
                    triharmonic: bool = False, auto_shift: bool = False) -> int:
    L = lib()
    n = (C.c_int64 * dim)(*N)
    o = _opts(prec, 500, restart, 1, levels=levels, batch=batch, shift=shift, variable_beta=variable_beta,
              uhat_slots=uhat_slots, triharmonic=triharmonic, auto_shift=auto_shift)
    out = C.c_size_t(0)
    _check(L.ahoc_workspace_bytes(dim, n, C.byref(o), C.byref(out)), "ahoc_workspace_bytes")
    return int(out.value)


def _info_dict(info: "ahoc_info", st: int) -> Dict:
    return dict(iters=info.iters, restarts=info.restarts, rel_resid=info.rel_resid,
                ms_total=info.ms_total, ms_matvec=info.ms_matvec, status=st, launches=info.launches,
                kernel_ms={k: info.kernel_ms[i] for i, k in enumerate(KERNEL_NAMES)},
                kernel_launches={k: info.kernel_launches[i] for i, k in enumerate(KERNEL_NAMES)},
                levels=info.levels, coarse_iters=info.coarse_iters,
                kernel_ms_top={k: info.kernel_ms_top[i] for i, k in enumerate(KERNEL_NAMES)},
                kernel_launches_top={k: info.kernel_launches_top[i] for i, k in enumerate(KERNEL_NAMES)},
                refine_steps=info.refine_steps,
                refine_hist=[info.refine_hist[i] for i in range(min(16, info.refine_steps + 1))],
                inner_iters=[info.inner_iters[i] for i in range(min(16, info.refine_steps))],
                refine_du=[info.refine_du[i] for i in range(min(16, info.refine_steps))],
                vsolve_iters=info.vsolve_iters)


class Plan:
    """A solver plan for one grid shape and ``batch`` problems of it (``ahoc_plan_create``).

    With batch > 1, alpha, the boundary data, f and u hold ``batch`` arrays
    of their single-problem size back to back, and ``solve`` returns one info
    dict per problem.  The device workspace is a torch uint8 tensor handed to
    the library, so device memory comes from PyTorch's allocator.
    """

    def __init__(self, dim: int, N: Sequence[int], alpha: Optional[torch.Tensor], lo=None, hi=None,
                 g_D=None, g_N=None, lapt_gD=None, v_edge=None, g_L=None, navier: int = 0, shift: float = 0.0,
                 beta=None, triharmonic: bool = False, lap_gD=None, bilap=None, g_NN=None, lapt_w=None,
                 device=None, auto_shift: bool = False,
                 prec: int = AHOC_FP64,
                 max_iters: int = 500, restart: int = 100, precond: int = 1, stream=None, timing: bool = False,
                 levels: int = -1, refine_tol: float = 0.0, coarse_tol: float = 0.0, batch: int = 1,
                 graphs: bool = True, uhat_slots: int = 0, fused: bool = True, first32: bool = False):
        L = lib()
        self.dim = dim
        self.batch = int(batch)
        self.N = [int(n) for n in N]
        self.lo = list(lo) if lo is not None else [0.0] * dim
        self.hi = list(hi) if hi is not None else [1.0] * dim
        self.nfull = 1
        self.nint = 1
        for n in self.N:
            self.nfull *= n + 1
            self.nint *= n - 1
        self.ngamma = 0
        for a in range(dim):
            s = 1
            for b in range(dim):
                if b != a:
                    s *= self.N[b] - 1
            self.ngamma += 2 * s
        prec = _prec(prec)
        self.prec = prec
        self.device = alpha.device if alpha is not None else torch.device(device or "cuda")
        B = self.batch
        variable_beta = beta is not None and not auto_shift
        nb = workspace_bytes(dim, self.N, restart, prec, levels, B, shift, variable_beta, uhat_slots, triharmonic,
                             auto_shift)
        self.workspace_bytes = nb
        self._ws = torch.empty(nb, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        bd = ahoc_bdata(_ptr(g_D, B * self.nfull, "g_D"), _ptr(g_N, B * self.ngamma, "g_N"),
                        _ptr(lapt_gD, B * self.ngamma, "lapt_gD"), _ptr(v_edge, B * self.nfull, "v_edge"),
                        _ptr(g_L, B * self.ngamma, "g_L"), _ptr(beta, B * self.nfull, "beta"),
                        _ptr(lap_gD, B * self.nfull, "lap_gD"), _ptr(bilap, B * self.nfull, "bilap"),
                        _ptr(g_NN, B * self.ngamma, "g_NN"), _ptr(lapt_w, B * self.ngamma, "lapt_w"))
        o = _opts(prec, max_iters, restart, precond, self._ws, timing, levels, refine_tol, coarse_tol, B, graphs,
                  navier, shift, variable_beta, uhat_slots, fused, triharmonic, auto_shift, first32)
        h = C.c_void_p(0)
        n = (C.c_int64 * dim)(*self.N)
        lo_ = (C.c_double * dim)(*self.lo)
        hi_ = (C.c_double * dim)(*self.hi)
        _check(L.ahoc_plan_create(C.byref(h), dim, n, lo_, hi_, _ptr(alpha, B * self.nfull, "alpha"), C.byref(bd),
                                  C.byref(o), C.c_void_p(self.stream.cuda_stream)), "ahoc_plan_create")
        self._h = h
        assert L.ahoc_n_gamma(h) == self.ngamma
        assert L.ahoc_batch(h) == B
        self.active = [1] * B

    # -- Algorithm 1 ---------------------------------------------------------
    def solve(self, f: torch.Tensor, u: Optional[torch.Tensor] = None, tol: float = 1e-12,
              check: bool = True, q0: Optional[torch.Tensor] = None):
        """u for f (one grid per problem of the plan); returns (u, info) with
        info a dict, or for a batched plan a list of dicts (None for problems
        not taking part).  q0: GMRES's initial Q, one face array per problem
        (``ahoc_solve_from``; FP64 plans)."""
        B = self.batch
        if u is None:
            u = torch.empty(B * self.nfull, dtype=torch.float64, device=self.device)
        infos = (ahoc_info * B)()
        if q0 is None:
            st = lib().ahoc_solve(self._h, _ptr(f, B * self.nfull, "f"), _ptr(u, B * self.nfull, "u"), float(tol),
                                  infos)
            name = "ahoc_solve"
        else:
            st = lib().ahoc_solve_from(self._h, _ptr(f, B * self.nfull, "f"), _ptr(q0, B * self.ngamma, "q0"),
                                       _ptr(u, B * self.nfull, "u"), float(tol), infos)
            name = "ahoc_solve_from"
        if check:
            _check(st, name)
        out = [_info_dict(infos[b], infos[b].status) if self.active[b] else None for b in range(B)]
        return u, (out[0] if B == 1 else out)

    def solve_host(self, f_host: torch.Tensor, u_host: torch.Tensor, tol: float = 1e-12, check: bool = True):
        """``ahoc_solve_host``: f and u in host memory (float64, contiguous;
        pinned for fast copies); returns the info as ``solve`` does."""
        B = self.batch
        infos = (ahoc_info * B)()
        st = lib().ahoc_solve_host(self._h, _hptr(f_host, B * self.nfull, "f_host"),
                                   _hptr(u_host, B * self.nfull, "u_host"), float(tol), infos)
        if check:
            _check(st, "ahoc_solve_host")
        out = [_info_dict(infos[b], infos[b].status) if self.active[b] else None for b in range(B)]
        return u_host, (out[0] if B == 1 else out)

    def load(self, b: int, alpha: torch.Tensor, g_D=None, g_N=None, lapt_gD=None, v_edge=None, g_L=None, beta=None):
        """Replace problem b's coefficient and boundary data (``ahoc_plan_load``)."""
        bd = ahoc_bdata(_ptr(g_D, self.nfull, "g_D"), _ptr(g_N, self.ngamma, "g_N"),
                        _ptr(lapt_gD, self.ngamma, "lapt_gD"), _ptr(v_edge, self.nfull, "v_edge"),
                        _ptr(g_L, self.ngamma, "g_L"), _ptr(beta, self.nfull, "beta"))
        _check(lib().ahoc_plan_load(self._h, int(b), _ptr(alpha, self.nfull, "alpha"), C.byref(bd)), "ahoc_plan_load")

    def set_active(self, mask: Sequence[int]):
        """Problems taking part in the next calls (``ahoc_set_active``)."""
        m = [1 if v else 0 for v in mask]
        if len(m) != self.batch:
            raise ValueError("mask needs %d entries" % self.batch)
        _check(lib().ahoc_set_active(self._h, (C.c_int * self.batch)(*m)), "ahoc_set_active")
        self.active = m

    def matvec(self, q: torch.Tensor, y: Optional[torch.Tensor] = None) -> torch.Tensor:
        n = self.batch * self.ngamma
        if y is None:
            y = torch.empty(n, dtype=torch.float64, device=self.device)
        _check(lib().ahoc_matvec(self._h, _ptr(q, n, "q"), _ptr(y, n, "y")), "ahoc_matvec")
        return y

    def schur_rhs(self, f: torch.Tensor, b: Optional[torch.Tensor] = None) -> torch.Tensor:
        n = self.batch * self.ngamma
        if b is None:
            b = torch.empty(n, dtype=torch.float64, device=self.device)
        _check(lib().ahoc_schur_rhs(self._h, _ptr(f, self.batch * self.nfull, "f"), _ptr(b, n, "b")),
               "ahoc_schur_rhs")
        return b

    def last_qv(self, with_v: bool = True):
        B = self.batch
        q = torch.empty(B * self.ngamma, dtype=torch.float64, device=self.device)
        v = torch.empty(B * self.nfull, dtype=torch.float64, device=self.device) if with_v else None
        _check(lib().ahoc_last_qv(self._h, _ptr(q, B * self.ngamma, "q"), _ptr(v, B * self.nfull, "v")),
               "ahoc_last_qv")
        return q, v

    # -- components -------------------------------------------------------------
    def dst1(self, x: torch.Tensor, axis: int, out: Optional[torch.Tensor] = None, scale: float = 1.0):
        if out is None:
            out = torch.empty_like(x)
        _check(lib().ahoc_dst1(self._h, int(axis), _ptr(x, self.nint, "x"), _ptr(out, self.nint, "out"),
                               float(scale)), "ahoc_dst1")
        return out

    def poisson(self, rhs: torch.Tensor, out: Optional[torch.Tensor] = None):
        if out is None:
            out = torch.empty_like(rhs)
        _check(lib().ahoc_poisson(self._h, _ptr(rhs, self.nint, "rhs"), _ptr(out, self.nint, "out")), "ahoc_poisson")
        return out

    def close(self):
        """Destroy the plan and release its workspace tensor."""
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(lib().ahoc_plan_destroy(self._h), "ahoc_plan_destroy")
            self._h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_for_triharmonic(data: Dict, device="cuda", **kw) -> "Plan":
    """Create a triharmonic plan from a sampled problem (``inputs.sample_triharmonic``):
    the faces not clamped are the simply supported faces of the plan's mask."""
    def dev(key):
        t = torch.as_tensor(data[key], dtype=torch.float64)
        return t.reshape(-1).contiguous().to(device)
    clamped = set(data.get("clamped") or ())
    supported = sum(1 << f for f in range(2 * data["dim"]) if f not in clamped)
    return Plan(data["dim"], data["N"], None, lo=data["lo"], hi=data["hi"], g_D=dev("g_D"), g_N=dev("g_N"),
                navier=supported, triharmonic=True, lap_gD=dev("lap_gD"), bilap=dev("bilap"), g_NN=dev("g_NN"),
                lapt_w=dev("lapt_w"), device=device, **kw)


def plan_for(data: Dict, device="cuda", **kw) -> "Plan":
    """Create a plan from a sampled problem (see ``paper_2609_16478_b300.inputs.sample``).

    The problem's Navier faces become the plan's mask; a nonzero beta (a
    number or a full-grid array) is passed as a full-grid array and the plan
    derives the beta class from it (``opts.auto_shift``: constant
    beta / alpha gives the shifted eigenvalues, otherwise the BiCGSTAB
    v-solves).
    """
    def dev(key):
        v = data.get(key)
        if v is None:
            return None
        t = torch.as_tensor(v, dtype=torch.float64)
        return t.reshape(-1).contiguous().to(device)
    alpha = dev("alpha")
    navier = sum(1 << int(f) for f in (data.get("navier") or ()))
    beta = data.get("beta")
    if beta is not None and (np.ndim(beta) > 0 or float(beta) != 0.0):
        if np.ndim(beta) > 0:
            kw.setdefault("beta", dev("beta"))
        else:
            kw.setdefault("beta", torch.full_like(alpha, float(beta)))
        kw.setdefault("auto_shift", True)
    kw.setdefault("navier", navier)
    return Plan(data["dim"], data["N"], alpha, lo=data["lo"], hi=data["hi"], g_D=dev("g_D"),
                g_N=dev("g_N"), lapt_gD=dev("lapt_gD"), v_edge=dev("v_edge"), g_L=dev("g_L"), **kw)
