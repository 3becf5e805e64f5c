"""Python binding of libphisplit.so (include/phisplit.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module converts torch
tensors to device pointers and sizes, keeps arrays referenced by the plan's
descriptors alive, and turns negative status codes into exceptions.  There is no
fallback: if the shared library is missing or fails to load, every call raises.

Layouts follow the library: a state tensor of sizes n_1 x ... x n_d is a
contiguous float64 CUDA tensor of shape (n_d, ..., n_1) (i_1 fastest); a small
matrix M is passed column-major, i.e. as the contiguous tensor M^T.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional, Sequence

import numpy as np
import torch

from . import workloads as wl

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libphisplit.so")

MM_OK = 0
MM_FP64, MM_TF32X3, MM_BF16X3 = 0, 1, 2
EXPEULER, ETD2RK, LAWSON_EULER, LAWSON2B, EXPROSEULER, EXPEULER_ALT = 0, 1, 2, 3, 4, 5
G_NONE, G_CUBIC, G_RICCATI, G_ADR_MANUFACTURED = 0, 1, 2, 3
STATUS_NONFINITE, STATUS_TIMEOUT = 1, 2
PRECISIONS = {"fp64": MM_FP64, "tf32x3": MM_TF32X3, "bf16x3": MM_BF16X3}

EXPORTS = ("phi_plan_create", "phi_plan_destroy", "phi_plan_info", "phi_plan_get_phi",
           "phi_plan_status", "mumode_workspace_bytes", "mumode_phi_apply",
           "expint_workspace_bytes", "expint_step", "phi_plan_set_graphs", "mm_status_str", "mm_version",
           "mm_trace_enable", "mm_trace_read", "tucker_apply_noalloc",
           "expint_batch_create", "expint_batch_run", "expint_batch_status", "expint_batch_info",
           "expint_batch_destroy", "expint_batched", "mm_batch_tile_plan", "expint_batch_schedule",
           "expint_batch_tile_order",
           "expint_batch_set_graph")
KC_CONTRACT_FP64, KC_CONTRACT_TF32, KC_PREPASS, KC_SPLIT = 0, 1, 2, 3


class PhisplitError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {status_str(code)} ({code})")


class Nonlin(ctypes.Structure):
    """mm_nonlin of include/phisplit.h."""
    _fields_ = [("kind", ctypes.c_int), ("c", ctypes.c_double * 4),
                ("B", ctypes.c_void_p), ("C", ctypes.c_void_p),
                ("psi_a", ctypes.c_void_p), ("psi_b", ctypes.c_void_p)]


class Tune(ctypes.Structure):
    """mm_tune of include/phisplit.h."""
    _fields_ = [("autotune", ctypes.c_int), ("nc_cap", ctypes.c_int), ("graph", ctypes.c_int)]


_lib = None


def lib():
    """Load libphisplit.so (raises if it is missing: build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                           "(the CUDA library has no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, f64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    L.phi_plan_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(i64), ctypes.POINTER(vp),
                                  f64, i32, i32, vp]
    L.phi_plan_destroy.argtypes = [vp]
    L.phi_plan_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32),
                                ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.phi_plan_get_phi.argtypes = [vp, i32, i32, vp, vp]
    L.phi_plan_status.argtypes = [vp, i32, vp]
    L.mumode_workspace_bytes.argtypes = [vp]
    L.mumode_workspace_bytes.restype = sz
    L.mumode_phi_apply.argtypes = [vp, i32, vp, vp, f64, vp, sz, vp]
    L.expint_workspace_bytes.argtypes = [vp, i32, ctypes.POINTER(Nonlin)]
    L.expint_workspace_bytes.restype = sz
    L.expint_step.argtypes = [vp, i32, ctypes.POINTER(Nonlin), vp, f64, i32, vp, sz, vp]
    L.phi_plan_set_graphs.argtypes = [vp, i32]
    L.mm_status_str.argtypes = [i32]
    L.mm_status_str.restype = ctypes.c_char_p
    L.mm_version.argtypes = []
    L.tucker_apply_noalloc.argtypes = [i32, ctypes.POINTER(i64), ctypes.POINTER(vp), vp, vp, f64, vp]
    P = ctypes.POINTER
    L.expint_batch_create.argtypes = [P(vp), i32, P(vp), P(Nonlin), P(vp), i32, P(Tune), vp]
    L.expint_batch_run.argtypes = [vp, f64, i32, vp]
    L.expint_batch_status.argtypes = [vp, i32, vp]
    L.expint_batch_info.argtypes = [vp, P(i32), P(i32), P(i64), P(i64)]
    L.expint_batch_destroy.argtypes = [vp]
    L.expint_batch_schedule.argtypes = [vp, P(ctypes.c_int32), i32, P(i32), P(ctypes.c_float), P(ctypes.c_float)]
    L.expint_batch_tile_order.argtypes = [vp]
    L.expint_batch_set_graph.argtypes = [vp, i32]
    L.expint_batched.argtypes = [i32, P(vp), P(Nonlin), P(vp), i32, f64, i32, P(Tune), vp]
    L.mm_batch_tile_plan.argtypes = [i32, P(i64), P(i64), i32, i32, i32, P(ctypes.c_int32), i64, P(i64)]
    L.mm_trace_enable.argtypes = [i32]
    L.mm_trace_read.argtypes = [i32, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(f64)]
    for name in EXPORTS:
        getattr(L, name).restype = getattr(L, name).restype or ctypes.c_int
    _lib = L
    return L


def status_str(code: int) -> str:
    try:
        return lib().mm_status_str(int(code)).decode()
    except Exception:
        return "unknown"


def _check(code: int, what: str) -> int:
    if code < 0:
        raise PhisplitError(code, what)
    return code


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return t.data_ptr()


def matrix_to_device(M, device="cuda") -> torch.Tensor:
    """Column-major device copy of an n x n matrix (returned as the tensor M^T)."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(M, dtype=np.float64).T)).to(device)


def matrix_from_device(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().T.copy()


class Plan:
    """phi_plan_create / phi_plan_destroy (Section 3.1 set-up)."""

    def __init__(self, A: Sequence, tau: float, ell_max: int = 2, prec: str = "fp64", stream=None):
        L = lib()
        self.A_dev = [a if isinstance(a, torch.Tensor) else matrix_to_device(a) for a in A]
        self.d = len(self.A_dev)
        self.n = [int(a.shape[0]) for a in self.A_dev]
        self.N = int(np.prod(self.n))
        self.tau = float(tau)
        self.ell_max = int(ell_max)
        self.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        n_arr = (ctypes.c_int64 * self.d)(*self.n)
        a_arr = (ctypes.c_void_p * self.d)(*[_ptr(a) for a in self.A_dev])
        h = ctypes.c_void_p()
        _check(L.phi_plan_create(ctypes.byref(h), self.d, n_arr, a_arr, self.tau, self.ell_max,
                                 self.prec, _stream(stream)), "phi_plan_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().phi_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        d = ctypes.c_int()
        n = (ctypes.c_int64 * self.d)()
        lm, pr, tri = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        sq = (ctypes.c_int * self.d)()
        _check(lib().phi_plan_info(self.handle, ctypes.byref(d), n, ctypes.byref(lm), ctypes.byref(pr),
                                   sq, ctypes.byref(tri)), "phi_plan_info")
        return {"d": d.value, "n": list(n), "ell_max": lm.value, "prec": pr.value,
                "squarings": list(sq), "tridiagonal": bool(tri.value)}

    def get_phi(self, ell: int, mu: int) -> np.ndarray:
        n = self.n[mu - 1]
        out = torch.empty((n, n), dtype=torch.float64, device="cuda")
        _check(lib().phi_plan_get_phi(self.handle, ell, mu, _ptr(out), _stream()), "phi_plan_get_phi")
        return matrix_from_device(out)

    def status(self, reset: bool = True) -> int:
        return _check(lib().phi_plan_status(self.handle, int(reset), _stream()), "phi_plan_status")

    def set_graphs(self, on: bool) -> None:
        """expint_step replays captured CUDA graphs (default) or launches directly."""
        _check(lib().phi_plan_set_graphs(self.handle, int(on)), "phi_plan_set_graphs")


def mumode_workspace(plan: Plan) -> torch.Tensor:
    nbytes = lib().mumode_workspace_bytes(plan.handle)
    return torch.empty(max(1, (nbytes + 7) // 8), dtype=torch.float64, device="cuda")


def mumode_phi_apply(plan: Plan, ell: int, V: torch.Tensor, P: Optional[torch.Tensor] = None,
                     alpha: float = 1.0, ws: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """P = alpha (l!)^(d-1) V x_1 phi_l(tau A_1) ... x_d phi_l(tau A_d)  (Section 3)."""
    if P is None:
        P = torch.empty_like(V)
    if ws is None:
        ws = mumode_workspace(plan)
    _check(lib().mumode_phi_apply(plan.handle, int(ell), _ptr(V), _ptr(P), float(alpha),
                                  _ptr(ws), ws.numel() * 8, _stream(stream)), "mumode_phi_apply")
    return P


class Nonlinearity:
    """mm_nonlin plus the device arrays it points to (kept alive here)."""

    def __init__(self, kind: int = G_NONE, cubic=(0.0, 0.0, 0.0, 0.0), B=None, C=None,
                 psi_a=None, psi_b=None):
        self.keep = []

        def dev(x, colmajor=False):
            if x is None:
                return None
            if isinstance(x, torch.Tensor):
                t = x
            elif colmajor:
                t = matrix_to_device(x)
            else:
                t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
            self.keep.append(t)
            return _ptr(t)

        self.struct = Nonlin()
        self.struct.kind = int(kind)
        for i in range(4):
            self.struct.c[i] = float(cubic[i])
        self.struct.B = dev(B, colmajor=True)
        self.struct.C = dev(C)          # already stored in state layout (n_2, n_1)
        self.struct.psi_a = dev(psi_a)
        self.struct.psi_b = dev(psi_b)

    @classmethod
    def from_problem(cls, p: "wl.Problem") -> "Nonlinearity":
        return cls(p.g_kind, p.cubic, p.B, p.C, p.psi_a, p.psi_b)


def expint_workspace(plan: Plan, scheme: int, g: Optional[Nonlinearity] = None) -> torch.Tensor:
    gs = ctypes.byref(g.struct) if g is not None else None
    nbytes = lib().expint_workspace_bytes(plan.handle, int(scheme), gs)
    return torch.empty(max(1, (nbytes + 7) // 8), dtype=torch.float64, device="cuda")


def expint_step(plan: Plan, scheme: int, U: torch.Tensor, nsteps: int, t0: float = 0.0,
                g: Optional[Nonlinearity] = None, ws: Optional[torch.Tensor] = None,
                stream=None) -> torch.Tensor:
    """Advance U in place by nsteps PHISPLIT steps (Section 3.2)."""
    if ws is None:
        ws = expint_workspace(plan, scheme, g)
    gs = ctypes.byref(g.struct) if g is not None else None
    _check(lib().expint_step(plan.handle, int(scheme), gs, _ptr(U), float(t0), int(nsteps),
                             _ptr(ws), ws.numel() * 8, _stream(stream)), "expint_step")
    return U


def trace_enable(on: bool = True) -> None:
    """Start a new tracing window (counts always; event timing if on)."""
    lib().mm_trace_enable(int(on))


def trace_read(cls: int, timed: bool = True):
    """(launches, device ms) of kernel class cls in the current window."""
    n = ctypes.c_longlong()
    ms = ctypes.c_double()
    _check(lib().mm_trace_read(int(cls), ctypes.byref(n), ctypes.byref(ms) if timed else None),
           "mm_trace_read")
    return n.value, (ms.value if timed else None)


def ell_for_scheme(scheme: int) -> int:
    return {EXPEULER: 1, ETD2RK: 2, LAWSON_EULER: 0, LAWSON2B: 0, EXPROSEULER: 1, EXPEULER_ALT: 1}[scheme]


def setup(problem: "wl.Problem", prec: str = "fp64", ell_max: Optional[int] = None):
    """Device plan, nonlinearity and initial state of a workloads.Problem."""
    ell = ell_for_scheme(problem.scheme) if ell_max is None else ell_max
    plan = Plan(problem.A, problem.tau, ell, prec)
    g = Nonlinearity.from_problem(problem)
    U = torch.from_numpy(np.ascontiguousarray(problem.u0)).cuda()
    return plan, g, U


class Batch:
    """expint_batch_create / run / destroy: many independent 2D problems stepped
    together in a mixed form (one graph launch per run)."""

    def __init__(self, plans: Sequence[Plan], gs: Optional[Sequence[Optional[Nonlinearity]]],
                 Us: Sequence[torch.Tensor], scheme: int = EXPEULER, autotune: bool = True,
                 nc_cap: int = 0, graph: bool = True, stream=None):
        L = lib()
        self.plans = list(plans)
        self.Us = list(Us)
        self.gs = list(gs) if gs is not None else None
        n = len(self.plans)
        h_arr = (ctypes.c_void_p * n)(*[p.handle.value for p in self.plans])
        u_arr = (ctypes.c_void_p * n)(*[_ptr(u) for u in self.Us])
        g_arr = None
        if self.gs is not None:
            g_arr = (Nonlin * n)()
            for j, g in enumerate(self.gs):
                if g is not None:
                    g_arr[j] = g.struct
        self.tune = Tune(int(autotune), int(nc_cap), int(graph))
        h = ctypes.c_void_p()
        _check(L.expint_batch_create(ctypes.byref(h), n, h_arr, g_arr, u_arr, int(scheme),
                                     ctypes.byref(self.tune), _stream(stream)), "expint_batch_create")
        self.handle = h

    def run(self, nsteps: int, t0: float = 0.0, stream=None) -> None:
        _check(lib().expint_batch_run(self.handle, float(t0), int(nsteps), _stream(stream)),
               "expint_batch_run")

    def status(self, reset: bool = True) -> int:
        return _check(lib().expint_batch_status(self.handle, int(reset), _stream()), "expint_batch_status")

    def info(self) -> dict:
        nc, cap = ctypes.c_int(), ctypes.c_int()
        t, dof = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().expint_batch_info(self.handle, ctypes.byref(nc), ctypes.byref(cap), ctypes.byref(t),
                                       ctypes.byref(dof)), "expint_batch_info")
        return {"classes": nc.value, "nc_cap": cap.value, "tiles_mode1": t.value, "dof": dof.value}

    def schedule(self) -> dict:
        """The autotuner's outcome: per-class tile widths, the Tucker time of a step
        with the best uniform width and with the schedule in use, and the tile order."""
        n = self.info()["classes"]
        w = (ctypes.c_int32 * max(n, 1))()
        nc, mu, mc = ctypes.c_int(), ctypes.c_float(), ctypes.c_float()
        per = _check(lib().expint_batch_schedule(self.handle, w, n, ctypes.byref(nc), ctypes.byref(mu),
                                                 ctypes.byref(mc)), "expint_batch_schedule")
        order = _check(lib().expint_batch_tile_order(self.handle), "expint_batch_tile_order")
        return {"per_class": bool(per), "widths": list(w)[:n], "tucker_ms_uniform": mu.value,
                "tucker_ms_chosen": mc.value,
                "tile_order": "alternate rounds reversed" if order == 1 else "round-robin"}

    def set_graph(self, on: bool) -> None:
        """Replay captured graphs (default) or launch the kernels directly."""
        _check(lib().expint_batch_set_graph(self.handle, int(on)), "expint_batch_set_graph")

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().expint_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_tile_plan(n1: Sequence[int], n2: Sequence[int], prec: str = "bf16x3", nc_cap: int = 128,
                    mode: int = 1) -> np.ndarray:
    """Host-only tile list of a batch (mm_batch_tile_plan): rows {instance, row tile,
    column split, size class}, in launch order."""
    L = lib()
    cnt = len(n1)
    a1 = (ctypes.c_int64 * cnt)(*[int(v) for v in n1])
    a2 = (ctypes.c_int64 * cnt)(*[int(v) for v in n2])
    nt = ctypes.c_int64()
    _check(L.mm_batch_tile_plan(cnt, a1, a2, PRECISIONS[prec], int(nc_cap), int(mode), None, 0,
                                ctypes.byref(nt)), "mm_batch_tile_plan")
    buf = (ctypes.c_int32 * (4 * nt.value))()
    _check(L.mm_batch_tile_plan(cnt, a1, a2, PRECISIONS[prec], int(nc_cap), int(mode), buf, nt.value,
                                ctypes.byref(nt)), "mm_batch_tile_plan")
    return np.frombuffer(buf, dtype=np.int32).reshape(-1, 4).copy()


def flat_offsets(problems: Sequence["wl.Problem"]):
    """Offsets (in doubles) of the states packed one after the other, each starting on a
    16-byte boundary, and the total length."""
    offs, o = [], 0
    for p in problems:
        offs.append(o)
        o += (p.u0.size + 1) // 2 * 2
    return offs, o


def setup_batch(problems: Sequence["wl.Problem"], prec: str = "bf16x3", flat: bool = False):
    """Plans, nonlinearities and device states of a list of independent problems.  With
    flat=True the states are views of one device buffer (packed by flat_offsets, so one
    copy moves them all), returned as a fourth value."""
    plans, gs, Us = [], [], []
    for p in problems:
        plans.append(Plan(p.A, p.tau, ell_for_scheme(p.scheme), prec))
        gs.append(Nonlinearity.from_problem(p))
    if not flat:
        Us = [torch.from_numpy(np.ascontiguousarray(p.u0)).cuda() for p in problems]
        return plans, gs, Us
    Us, buf = flat_states(problems)
    return plans, gs, Us, buf


def flat_states(problems: Sequence["wl.Problem"]):
    """The problems' initial states as views of one device buffer (flat_offsets), and
    the buffer."""
    offs, total = flat_offsets(problems)
    buf = torch.zeros(total, dtype=torch.float64, device="cuda")
    Us = []
    for p, o in zip(problems, offs):
        u = buf[o:o + p.u0.size].view(p.u0.shape)
        u.copy_(torch.from_numpy(np.ascontiguousarray(p.u0)))
        Us.append(u)
    return Us, buf
