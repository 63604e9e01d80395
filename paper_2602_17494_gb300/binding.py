"""Thin ctypes binding of libtvs (declarations in include/tvs.h).

Argument marshalling only: torch tensors supply device pointers and the
current CUDA stream; every step of the method runs in the library's kernels.
Importing this module loads ``libtvs.so`` and raises if it is missing -- there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtvs.so")

TVS_OK = 0
TVS_ERR_NOT_CONVERGED = 5
TVS_F32, TVS_BF16, TVS_F16, TVS_S16 = 0, 1, 2, 3


class TvsIter(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int), ("t", ctypes.c_double), ("rel_gap_tol", ctypes.c_double),
                ("check_every", ctypes.c_int), ("storage", ctypes.c_int)]


class TvsReport(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("dual_D", ctypes.c_double), ("primal_E", ctypes.c_double),
                ("gap", ctypes.c_double), ("rel_gap", ctypes.c_double), ("div_res_max", ctypes.c_double),
                ("max_p", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class TvsDecomp(ctypes.Structure):
    _fields_ = [("m2", ctypes.c_int), ("m1", ctypes.c_int), ("overlap", ctypes.c_int),
                ("k_inner", ctypes.c_int), ("alpha_hat", ctypes.c_double)]


class TvsEngineConfig(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("alpha", ctypes.c_double), ("eps", ctypes.c_double),
                ("it1", TvsIter), ("it2", TvsIter), ("tile", ctypes.c_int), ("overlap", ctypes.c_int),
                ("k_inner", ctypes.c_int), ("max_live", ctypes.c_int)]


class TvsError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib.tvs_status_string(status).decode()
        extra = _lib.tvs_last_error().decode()
        super().__init__(f"{where}: {msg} (status {status}){': ' + extra if extra else ''}")
        self.status = status


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libtvs.so not built ({LIB_PATH}); run paper_2602_17494_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    lib.tvs_version.restype = I
    lib.tvs_status_string.restype = ctypes.c_char_p
    lib.tvs_status_string.argtypes = [I]
    lib.tvs_last_error.restype = ctypes.c_char_p
    lib.tvs_workspace_bytes.restype = S
    lib.tvs_workspace_bytes.argtypes = [I, I, I, ctypes.POINTER(TvsDecomp), I]
    lib.tvs_project.restype = I
    lib.tvs_project.argtypes = [P, P, I, I, P, S, P]
    lib.tvs_step1.restype = I
    lib.tvs_step1.argtypes = [P, I, I, D, ctypes.POINTER(TvsIter), P, P, P, S, P, ctypes.POINTER(TvsReport)]
    lib.tvs_step2.restype = I
    lib.tvs_step2.argtypes = [P, P, I, I, D, D, ctypes.POINTER(TvsIter), P, P, P, S, P,
                              ctypes.POINTER(TvsReport)]
    lib.tvs_denoise.restype = I
    lib.tvs_denoise.argtypes = [P, I, I, D, D, D, ctypes.POINTER(TvsIter), ctypes.POINTER(TvsIter),
                                ctypes.POINTER(TvsDecomp), P, P, P, S, P, ctypes.POINTER(TvsReport)]
    lib.tvs_schwarz.restype = I
    lib.tvs_schwarz.argtypes = [I, P, P, I, I, D, D, ctypes.POINTER(TvsDecomp), ctypes.POINTER(TvsIter),
                                P, P, P, S, P, ctypes.POINTER(TvsReport)]
    lib.tvs_step2_w11.restype = I
    lib.tvs_step2_w11.argtypes = [P, P, I, I, D, D, ctypes.POINTER(TvsIter), P, P, P, P, S, P,
                                  ctypes.POINTER(TvsReport)]
    lib.tvs_irv2.restype = I
    lib.tvs_irv2.argtypes = [P, P, I, I, D, ctypes.POINTER(TvsIter), ctypes.POINTER(TvsDecomp), P, P, P, P, S, P,
                             ctypes.POINTER(TvsReport)]
    lib.tvs_project_noalloc.restype = I
    lib.tvs_project_noalloc.argtypes = [P, P, I, I, P]
    lib.tvs_profile_enable.restype = I
    lib.tvs_profile_enable.argtypes = [I]
    lib.tvs_set_wait_limit.restype = I
    lib.tvs_set_wait_limit.argtypes = [ctypes.c_longlong]
    lib.tvs_set_graphs.restype = I
    lib.tvs_set_graphs.argtypes = [I]
    lib.tvs_profile_read.restype = I
    lib.tvs_profile_read.argtypes = [ctypes.POINTER(TvsKernelTime), I]
    E = ctypes.POINTER(TvsEngineConfig)
    lib.tvs_engine_request_bytes.restype = S
    lib.tvs_engine_request_bytes.argtypes = [E, I, I]
    lib.tvs_engine_pool_overhead.restype = S
    lib.tvs_engine_pool_overhead.argtypes = [E]
    lib.tvs_engine_create.restype = I
    lib.tvs_engine_create.argtypes = [E, P, S, P, ctypes.POINTER(P)]
    lib.tvs_engine_submit.restype = I
    lib.tvs_engine_submit.argtypes = [P, ctypes.c_longlong, P, I, I, P]
    lib.tvs_engine_step.restype = I
    lib.tvs_engine_step.argtypes = [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(TvsReport), I,
                                    ctypes.POINTER(I)]
    lib.tvs_engine_pending.restype = I
    lib.tvs_engine_pending.argtypes = [P]
    lib.tvs_engine_destroy.restype = None
    lib.tvs_engine_destroy.argtypes = [P]
    lib.tvs_quality.restype = I
    lib.tvs_quality.argtypes = [P, P, I, I, P, S, P, ctypes.POINTER(D), ctypes.POINTER(D)]
    IP = ctypes.POINTER(I)
    lib.tvs_tune_workspace_bytes.restype = S
    lib.tvs_tune_workspace_bytes.argtypes = [I, I, IP, I, IP, I, I]
    lib.tvs_tune_schwarz2.restype = I
    lib.tvs_tune_schwarz2.argtypes = [P, P, I, I, D, D, ctypes.POINTER(TvsIter), IP, I, IP, I, IP, I, P, S, P, IP,
                                      ctypes.POINTER(ctypes.c_float)]
    return lib


class TvsKernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int), ("ms", ctypes.c_double)]


_lib = _load()

# Every symbol that include/tvs.h declares.
EXPORTED = ["tvs_denoise", "tvs_engine_create", "tvs_engine_destroy", "tvs_engine_pending",
            "tvs_engine_pool_overhead", "tvs_engine_request_bytes", "tvs_engine_step", "tvs_engine_submit",
            "tvs_last_error", "tvs_profile_enable", "tvs_profile_read", "tvs_project",
            "tvs_project_noalloc", "tvs_quality", "tvs_schwarz", "tvs_set_graphs", "tvs_set_wait_limit", "tvs_status_string", "tvs_step1",
            "tvs_step2", "tvs_step2_w11", "tvs_irv2",
            "tvs_tune_schwarz2", "tvs_tune_workspace_bytes", "tvs_version",
            "tvs_workspace_bytes"]


def lib() -> ctypes.CDLL:
    return _lib


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("libtvs takes contiguous float32 CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _check(st: int, where: str, allow_not_converged: bool = True):
    if st == TVS_OK or (allow_not_converged and st == TVS_ERR_NOT_CONVERGED):
        return
    raise TvsError(st, where)


def make_iter(max_iter: int, t: float = 0.125, rel_gap_tol: float = 0.0, check_every: int = 0,
              storage: int = TVS_F32) -> TvsIter:
    return TvsIter(int(max_iter), float(t), float(rel_gap_tol), int(check_every), int(storage))


def make_decomp(m2: int, m1: int, overlap: int, k_inner: int, alpha_hat: float = 0.0) -> TvsDecomp:
    return TvsDecomp(int(m2), int(m1), int(overlap), int(k_inner), float(alpha_hat))


def workspace_bytes(step: int, n2: int, n1: int, dd: TvsDecomp | None = None, storage: int = TVS_F32) -> int:
    n = _lib.tvs_workspace_bytes(step, n2, n1, ctypes.byref(dd) if dd is not None else None, storage)
    if n == 0:
        raise ValueError(f"unsupported sizes for step {step}: {n2} x {n1}")
    return int(n)


def workspace(step: int, n2: int, n1: int, dd: TvsDecomp | None = None, device=None,
              storage: int = TVS_F32) -> torch.Tensor:
    n = workspace_bytes(step, n2, n1, dd, storage)
    return torch.empty(n, dtype=torch.uint8, device=device or "cuda")


@dataclass
class Result:
    out: torch.Tensor
    report: dict
    status: int


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def tvs_project(tau: torch.Tensor, out: torch.Tensor | None = None, ws: torch.Tensor | None = None) -> torch.Tensor:
    """P_K of a 2-plane field of shape (2, rows, cols)."""
    _, rows, cols = tau.shape
    out = torch.empty_like(tau) if out is None else out
    ws = workspace(3, rows - 1, cols - 1, device=tau.device) if ws is None else ws
    st = _lib.tvs_project(_ptr(tau), _ptr(out), rows, cols, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                          _stream(tau.device))
    _check(st, "tvs_project", False)
    return out


def tvs_project_noalloc(tau: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """P_K without a workspace (fixed internal scratch, grids up to 1025 x 1025)."""
    _, rows, cols = tau.shape
    out = torch.empty_like(tau) if out is None else out
    st = _lib.tvs_project_noalloc(_ptr(tau), _ptr(out), rows, cols, _stream(tau.device))
    _check(st, "tvs_project_noalloc", False)
    return out


def tvs_step1(d0: torch.Tensor, delta: float, it: TvsIter, tau: torch.Tensor | None = None,
              p: torch.Tensor | None = None, ws: torch.Tensor | None = None) -> Result:
    n2, n1 = d0.shape
    tau = torch.empty((2, n2 + 1, n1 + 1), dtype=torch.float32, device=d0.device) if tau is None else tau
    ws = workspace(1, n2, n1, device=d0.device, storage=it.storage) if ws is None else ws
    rep = TvsReport()
    st = _lib.tvs_step1(_ptr(d0), n2, n1, float(delta), ctypes.byref(it), _ptr(tau), _ptr(p),
                        ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(d0.device), ctypes.byref(rep))
    _check(st, "tvs_step1")
    return Result(tau, rep.as_dict(), st)


def tvs_step2(d0: torch.Tensor, tau: torch.Tensor, alpha: float, eps: float, it: TvsIter,
              d: torch.Tensor | None = None, p: torch.Tensor | None = None,
              ws: torch.Tensor | None = None) -> Result:
    n2, n1 = d0.shape
    d = torch.empty_like(d0) if d is None else d
    ws = workspace(2, n2, n1, device=d0.device, storage=it.storage) if ws is None else ws
    rep = TvsReport()
    st = _lib.tvs_step2(_ptr(d0), _ptr(tau), n2, n1, float(alpha), float(eps), ctypes.byref(it), _ptr(d), _ptr(p),
                        ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(d0.device), ctypes.byref(rep))
    _check(st, "tvs_step2")
    return Result(d, rep.as_dict(), st)


def tvs_step2_w11(d0: torch.Tensor, tau: torch.Tensor, alpha: float, eps: float, it: TvsIter,
                  d: torch.Tensor | None = None, p: torch.Tensor | None = None, p0: torch.Tensor | None = None,
                  ws: torch.Tensor | None = None):
    """W^{1,1} step 2: returns (d, p, report, status) with p the dual of eq. IRW11:dual."""
    n2, n1 = d0.shape
    d = torch.empty_like(d0) if d is None else d
    p = torch.empty((2, n2, n1), dtype=torch.float32, device=d0.device) if p is None else p
    ws = workspace(2, n2, n1, device=d0.device, storage=it.storage) if ws is None else ws
    rep = TvsReport()
    st = _lib.tvs_step2_w11(_ptr(d0), _ptr(tau), n2, n1, float(alpha), float(eps), ctypes.byref(it), _ptr(d),
                            _ptr(p), _ptr(p0), ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(d0.device),
                            ctypes.byref(rep))
    _check(st, "tvs_step2_w11")
    return d, p, rep.as_dict(), st


def tvs_irv2(d0: torch.Tensor, tau: torch.Tensor, alpha: float, it: TvsIter, dd: TvsDecomp | None = None,
             d: torch.Tensor | None = None, p: torch.Tensor | None = None, g: torch.Tensor | None = None,
             ws: torch.Tensor | None = None):
    """IRV2 step 2: returns (d, g, report, status); g is the potential of tau_perp."""
    n2, n1 = d0.shape
    d = torch.empty_like(d0) if d is None else d
    g = torch.empty_like(d0) if g is None else g
    ws = workspace(5, n2, n1, dd, device=d0.device, storage=it.storage) if ws is None else ws
    rep = TvsReport()
    st = _lib.tvs_irv2(_ptr(d0), _ptr(tau), n2, n1, float(alpha), ctypes.byref(it),
                       ctypes.byref(dd) if dd is not None else None, _ptr(d), _ptr(p), _ptr(g),
                       ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(d0.device), ctypes.byref(rep))
    _check(st, "tvs_irv2")
    return d, g, rep.as_dict(), st


def tvs_denoise(d0: torch.Tensor, delta: float, alpha: float, eps: float, it1: TvsIter, it2: TvsIter,
                dd2: TvsDecomp | None = None, tau: torch.Tensor | None = None, d: torch.Tensor | None = None,
                ws: torch.Tensor | None = None):
    n2, n1 = d0.shape
    d = torch.empty_like(d0) if d is None else d
    ws = workspace(0, n2, n1, dd2, device=d0.device, storage=it2.storage) if ws is None else ws
    reps = (TvsReport * 2)()
    st = _lib.tvs_denoise(_ptr(d0), n2, n1, float(delta), float(alpha), float(eps), ctypes.byref(it1),
                          ctypes.byref(it2), ctypes.byref(dd2) if dd2 is not None else None, _ptr(tau), _ptr(d),
                          ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(d0.device), reps)
    _check(st, "tvs_denoise")
    return d, tau, [reps[0].as_dict(), reps[1].as_dict()], st


def tvs_schwarz(step: int, d0: torch.Tensor, tau: torch.Tensor | None, weight: float, eps: float,
                dd: TvsDecomp, outer: TvsIter, out: torch.Tensor | None = None, p: torch.Tensor | None = None,
                ws: torch.Tensor | None = None) -> Result:
    n2, n1 = d0.shape
    if out is None:
        shape = (n2, n1) if step == 2 else (2, n2 + 1, n1 + 1)
        out = torch.empty(shape, dtype=torch.float32, device=d0.device)
    ws = workspace(step, n2, n1, dd, device=d0.device, storage=outer.storage) if ws is None else ws
    rep = TvsReport()
    st = _lib.tvs_schwarz(step, _ptr(d0), _ptr(tau), n2, n1, float(weight), float(eps), ctypes.byref(dd),
                          ctypes.byref(outer), _ptr(out), _ptr(p), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                          _stream(d0.device), ctypes.byref(rep))
    _check(st, "tvs_schwarz")
    return Result(out, rep.as_dict(), st)


def tvs_set_wait_limit(cycles: int) -> None:
    """Limit of the bounded device-side waits in SM cycles (<= 0: the default)."""
    _check(_lib.tvs_set_wait_limit(int(cycles)), "tvs_set_wait_limit", False)


def tvs_set_graphs(on: bool) -> bool:
    """Turn graph replay of the iteration runs on or off; returns the previous setting."""
    return bool(_lib.tvs_set_graphs(1 if on else 0))


def tvs_profile_enable(on: bool = True) -> None:
    _lib.tvs_profile_enable(1 if on else 0)


def tvs_profile_read() -> dict:
    """{kernel class: (launches, summed device ms)} since the last enable."""
    buf = (TvsKernelTime * 16)()
    n = _lib.tvs_profile_read(buf, 16)
    return {buf[i].name.decode(): (buf[i].launches, buf[i].ms) for i in range(n)}


# ---------------------------------------------------------------------------
# batching / serving engine (tvs_engine_*)
# ---------------------------------------------------------------------------
def make_engine_config(delta: float, alpha: float, eps: float, it1: TvsIter, it2: TvsIter, tile: int = 64,
                       overlap: int = 4, k_inner: int = 16, max_live: int = 64) -> TvsEngineConfig:
    return TvsEngineConfig(float(delta), float(alpha), float(eps), it1, it2, int(tile), int(overlap), int(k_inner),
                           int(max_live))


class Engine:
    """Owns a device pool and a tvs_engine; requests are torch tensors on that device."""

    def __init__(self, cfg: TvsEngineConfig, pool_bytes: int, device=None):
        self.cfg = cfg
        self.device = torch.device(device or "cuda")
        over = _lib.tvs_engine_pool_overhead(ctypes.byref(cfg))
        if over == 0:
            raise ValueError("invalid engine configuration")
        self.pool = torch.empty(int(pool_bytes), dtype=torch.uint8, device=self.device)
        self.handle = ctypes.c_void_p()
        st = _lib.tvs_engine_create(ctypes.byref(cfg), ctypes.c_void_p(self.pool.data_ptr()), self.pool.numel(),
                                    _stream(self.device), ctypes.byref(self.handle))
        _check(st, "tvs_engine_create", False)
        self.requests = {}

    def request_bytes(self, n2: int, n1: int) -> int:
        return int(_lib.tvs_engine_request_bytes(ctypes.byref(self.cfg), n2, n1))

    def submit(self, rid: int, d0: torch.Tensor, d: torch.Tensor | None = None) -> torch.Tensor:
        n2, n1 = d0.shape
        d = torch.empty_like(d0) if d is None else d
        st = _lib.tvs_engine_submit(self.handle, int(rid), _ptr(d0), n2, n1, _ptr(d))
        _check(st, "tvs_engine_submit", False)
        self.requests[int(rid)] = (d0, d)     # keep the buffers alive until done
        return d

    def step(self, cap: int = 256):
        ids = (ctypes.c_longlong * max(cap, 1))()
        reps = (TvsReport * (2 * max(cap, 1)))()
        n = ctypes.c_int()
        st = _lib.tvs_engine_step(self.handle, ids, reps, cap, ctypes.byref(n))
        _check(st, "tvs_engine_step", False)
        out = []
        for k in range(n.value):
            d0, d = self.requests.pop(ids[k])
            out.append((ids[k], d, reps[2 * k].as_dict(), reps[2 * k + 1].as_dict()))
        return out

    def pending(self) -> int:
        return int(_lib.tvs_engine_pending(self.handle))

    def close(self) -> None:
        if self.handle:
            _lib.tvs_engine_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tvs_tune_schwarz2(d0: torch.Tensor, tau: torch.Tensor, alpha: float, eps: float, it: TvsIter,
                      tiles=(32, 48, 64), overlaps=(2, 4, 8), ks=(4, 8, 16)):
    """Fastest (tile, overlap, k) to it.rel_gap_tol on this image, and its milliseconds."""
    n2, n1 = d0.shape
    arr = lambda v: (ctypes.c_int * len(v))(*[int(x) for x in v])
    T, O, K = arr(tiles), arr(overlaps), arr(ks)
    need = _lib.tvs_tune_workspace_bytes(n2, n1, T, len(tiles), O, len(overlaps), it.storage)
    if need == 0:
        raise ValueError("no valid candidate decomposition")
    ws = torch.empty(int(need), dtype=torch.uint8, device=d0.device)
    best = (ctypes.c_int * 3)()
    ms = ctypes.c_float()
    st = _lib.tvs_tune_schwarz2(_ptr(d0), _ptr(tau), n2, n1, float(alpha), float(eps), ctypes.byref(it), T, len(tiles),
                                O, len(overlaps), K, len(ks), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                _stream(d0.device), best, ctypes.byref(ms))
    _check(st, "tvs_tune_schwarz2", False)
    return (best[0], best[1], best[2]), ms.value


def tvs_quality(d: torch.Tensor, gt: torch.Tensor, ws: torch.Tensor | None = None):
    """(PSNR, MSSIM) of d against gt (Section 5.3)."""
    n2, n1 = d.shape
    ws = workspace(4, max(n2, 2), max(n1, 2), device=d.device) if ws is None else ws
    ps, ms = ctypes.c_double(), ctypes.c_double()
    st = _lib.tvs_quality(_ptr(d), _ptr(gt), n2, n1, ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(d.device),
                          ctypes.byref(ps), ctypes.byref(ms))
    _check(st, "tvs_quality", False)
    return ps.value, ms.value
