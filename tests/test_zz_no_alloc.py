"""The allocation-free Tucker entry point, tucker_apply_noalloc.

It serves callers that may not allocate device memory when they need the split
action (an application that owns all device memory through its own pool, a loop
that cannot afford cudaMalloc's synchronisation, a plug-in barred from the CUDA
allocator).  It keeps its intermediate tensor in a fixed array built into the
library instead of a caller workspace.  This test calls it through the C ABI
twice in a row and checks each result against mumode_phi_apply, the entry point
that uses caller-provided workspace, and against the FP64 oracle's split action
(oracle.tucker.phisplit_apply with the oracle's own phi matrices), within the FP64
tolerance of the other parity tests (1e-12 relative).  The file is named to be
collected last.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from oracle.phi import phi_matrices
from oracle.tucker import phisplit_apply
from paper_2304_02327_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-12
MAX_ELEMS = 1 << 21      # MM_NOALLOC_MAX_ELEMS


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2304_02327_gb300 import api as _api, build
    build.build()
    _api.lib()
    return _api


def call_noalloc(api, plan, ell, V, alpha):
    """tucker_apply_noalloc with the plan's phi_ell matrices, through ctypes."""
    d = plan.d
    mats = []
    for mu in range(1, d + 1):
        n = plan.n[mu - 1]
        M = torch.empty((n, n), dtype=torch.float64, device="cuda")
        assert api.lib().phi_plan_get_phi(plan.handle, ell, mu, M.data_ptr(),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
        mats.append(M)
    P = torch.empty_like(V)
    n_arr = (ctypes.c_int64 * d)(*plan.n)
    m_arr = (ctypes.c_void_p * d)(*[M.data_ptr() for M in mats])
    scale = alpha * math.factorial(ell) ** (d - 1)
    rc = api.lib().tucker_apply_noalloc(d, n_arr, m_arr, V.data_ptr(), P.data_ptr(), scale,
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, api.status_str(rc)
    torch.cuda.synchronize()
    return P


def rel_err(a, b):
    return float((a - b).abs().max() / b.abs().max())


def oracle_apply(As, tau, ell, V, alpha):
    """alpha P_l^(2) V from the oracle's phi matrices (Pade route), as a tensor."""
    ref = alpha * phisplit_apply(V.cpu().numpy(), [phi_matrices(tau * A, ell)[ell] for A in As], ell)
    return torch.from_numpy(ref)


def test_noalloc_matches_workspace_entry_point_two_calls(api):
    # call 1: the 3D ADR operator at n = 128 (N = 2^21, the largest accepted size)
    p = wl.adr_3d(n=128, seed=2, steps=1)
    plan = api.Plan(p.A, p.tau, 2)
    V1 = torch.from_numpy(np.ascontiguousarray(p.u0)).cuda()
    got1 = call_noalloc(api, plan, 1, V1, 0.5)
    ref1 = api.mumode_phi_apply(plan, 1, V1, alpha=0.5)
    torch.cuda.synchronize()
    assert rel_err(got1, ref1) <= TOL
    orc1 = oracle_apply(p.A, p.tau, 1, V1, 0.5)
    assert rel_err(got1.cpu(), orc1) <= TOL
    # call 2 right after, different sizes, phi index and input: the shared
    # scratch still holds call 1's data and must not leak into the result
    ns = (37, 20, 9)
    As = [wl.fd_matrix(n, 0.3, 0.8) for n in ns]
    plan2 = api.Plan(As, 2e-3, 2)
    V2 = torch.from_numpy(wl.random_tensor(tuple(reversed(ns)), 11)).cuda()
    got2 = call_noalloc(api, plan2, 2, V2, -1.5)
    ref2 = api.mumode_phi_apply(plan2, 2, V2, alpha=-1.5)
    torch.cuda.synchronize()
    assert rel_err(got2, ref2) <= TOL
    assert rel_err(got2.cpu(), oracle_apply(As, 2e-3, 2, V2, -1.5)) <= TOL
    # and the first result is unchanged by the second call
    assert rel_err(got1, ref1) <= TOL
    assert rel_err(got1.cpu(), orc1) <= TOL


def test_noalloc_rejects_sizes_beyond_its_scratch(api):
    d = 3
    n_arr = (ctypes.c_int64 * d)(129, 128, 128)       # N > 2^21
    dummy = torch.empty(8, dtype=torch.float64, device="cuda")
    m_arr = (ctypes.c_void_p * d)(*([dummy.data_ptr()] * d))
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    rc = api.lib().tucker_apply_noalloc(d, n_arr, m_arr, dummy.data_ptr(), out.data_ptr(), 1.0, None)
    assert rc == -2                                     # MM_ERR_SHAPE, before any device work
