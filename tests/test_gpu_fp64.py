"""Parity of the plain FP64 CUDA path with the FP64 oracle (element by element).

Tolerance: the spec bar for the plain FP64 form is 1e-12 relative to the
oracle.  Both sides evaluate the same algorithm in double precision; they
differ only in summation order and in how phi_l(tau A_mu) is formed (the GPU
plan: Taylor + squaring eq. (16); the oracle: Pade-13 of an augmented matrix).
"""
import math

import numpy as np
import pytest
import torch

from oracle.integrators import OracleProblem, integrate, rel_err_inf, rel_err_fro
from oracle.phi import phi_matrices
from oracle.tucker import phisplit_apply
from paper_2304_02327_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2304_02327_gb300 import api as _api, build
    build.build()
    _api.lib()
    return _api


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


@pytest.mark.parametrize("n,eps,beta,tau,lmax", [
    (1, 0.3, 0.0, 1e-3, 2), (17, 0.5, 1.0, 1e-3, 2), (64, 0.01, 0.0, 1e-3, 1),
    (128, 0.5, 1.0, 1e-3, 2), (200, 0.75, 0.1, 0.025, 3), (48, 0.1, 0.0, 0.0, 2)])
def test_plan_phi_matches_oracle(api, n, eps, beta, tau, lmax):
    A = wl.fd_matrix(n, eps, beta)
    plan = api.Plan([A], tau, lmax)
    ref = phi_matrices(tau * A, lmax)
    for ell in range(lmax + 1):
        got = plan.get_phi(ell, 1)
        scale = max(1.0, np.abs(ref[ell]).max())
        assert np.abs(got - ref[ell]).max() <= 1e-13 * scale, (ell, np.abs(got - ref[ell]).max())


def test_plan_phi_dense_nonsymmetric(api):
    p = wl.riccati_2d(96, seed=3, tau=1e-3)
    plan = api.Plan(p.A, p.tau, 2)
    info = plan.info()
    assert not info["tridiagonal"]
    for mu in (1, 2):
        ref = phi_matrices(p.tau * p.A[mu - 1], 2)
        for ell in range(3):
            got = plan.get_phi(ell, mu)
            assert np.abs(got - ref[ell]).max() <= 1e-13 * max(1.0, np.abs(ref[ell]).max())


def test_plan_dedupes_equal_directions(api):
    A = wl.fd_matrix(33, 0.2)
    plan = api.Plan([A, A.copy(), wl.fd_matrix(33, 0.3)], 1e-2, 1)
    for ell in (0, 1):
        assert np.array_equal(plan.get_phi(ell, 1), plan.get_phi(ell, 2))
        assert not np.array_equal(plan.get_phi(ell, 1), plan.get_phi(ell, 3))


@pytest.mark.parametrize("ns", [(7,), (64, 64), (3, 5), (17, 48), (127, 33), (20, 17, 13),
                                (48, 64, 80), (1, 9, 4), (5, 4, 3, 6), (130, 3, 2)])
@pytest.mark.parametrize("ell", [0, 1, 2])
def test_mumode_phi_apply_matches_oracle(api, ns, ell):
    tau = 2e-3
    As = [wl.fd_matrix(n, 0.4, 0.9) + 0.05 * wl.random_dense(n, 100 + n) for n in ns]
    V = wl.random_tensor(tuple(reversed(ns)), seed=len(ns) * 7 + ell)
    plan = api.Plan(As, tau, 2)
    P = api.mumode_phi_apply(plan, ell, dev(V), alpha=0.7)
    ref = 0.7 * phisplit_apply(V, [phi_matrices(tau * A, 2)[ell] for A in As], ell)
    got = P.cpu().numpy()
    assert rel_err_inf(got, ref) <= TOL


def run_pair(api, p, prec="fp64"):
    plan, g, U = api.setup(p, prec)
    api.expint_step(plan, p.scheme, U, p.steps, g=g)
    torch.cuda.synchronize()
    assert plan.status() == 0
    ref = integrate(OracleProblem.from_problem(p), p.u0, p.scheme, p.steps)
    return U.cpu().numpy(), ref


@pytest.mark.parametrize("scheme", [wl.EXPEULER, wl.ETD2RK, wl.LAWSON_EULER, wl.LAWSON2B])
@pytest.mark.parametrize("sizes", [(24, 17, 13), (33, 40)])
def test_expint_schemes_match_oracle(api, scheme, sizes):
    if len(sizes) == 3:
        p = wl.adr_3d(seed=5, steps=4, scheme=scheme, sizes=sizes)
    else:
        p = wl.allen_cahn_2d(n=33, seed=6, steps=4, scheme=scheme)
        p.A = [wl.fd_matrix(33, 0.01), wl.fd_matrix(40, 0.02)]
        p.u0 = wl.random_tensor((40, 33), 6, -0.9, 0.9)
    got, ref = run_pair(api, p)
    assert rel_err_inf(got, ref) <= TOL


def test_expint_dense_operator_path(api):
    """Non-tridiagonal A_mu: K u runs as dense mode products."""
    ns = (21, 18)
    As = [wl.fd_matrix(n, 0.3, 0.2) + 0.3 * wl.random_dense(n, 7 + n) for n in ns]
    p = wl.Problem(name="dense", A=As, u0=wl.random_tensor((18, 21), 3), g_kind=wl.G_CUBIC,
                   cubic=(0.1, 1.0, 0.0, -1.0), tau=1e-2, steps=3, scheme=wl.ETD2RK)
    got, ref = run_pair(api, p)
    assert rel_err_inf(got, ref) <= TOL


@pytest.mark.parametrize("scheme", [wl.EXPEULER, wl.ETD2RK])
def test_riccati_small_matches_oracle(api, scheme):
    p = wl.riccati_2d(80, seed=9, tau=1e-4, steps=5, scheme=scheme)
    p.u0 = 0.01 * wl.random_tensor((80, 80), 4)
    got, ref = run_pair(api, p)
    assert rel_err_fro(got, ref) <= TOL and rel_err_inf(got, ref) <= TOL


def test_allen_cahn_n64_full_config(api):
    """2D Allen-Cahn, n = 64, eps = 0.01, 50 exponential Euler steps, FP64."""
    p = wl.workload("ac2d_n64_expeuler")
    got, ref = run_pair(api, p)
    assert rel_err_inf(got, ref) <= TOL


def test_adr3d_n128_full_config(api):
    """3D ADR, n = 128, 100 ETD2RK steps, FP64: the measured workload, full length."""
    p = wl.workload("adr3d_n128_etd2rk")
    got, ref = run_pair(api, p)
    assert rel_err_inf(got, ref) <= TOL and rel_err_fro(got, ref) <= TOL


def test_adr3d_n320_two_steps(api):
    """3D ADR at n = 320 (N = 32.8M), two ETD2RK steps in FP64 against the oracle."""
    p = wl.workload("adr3d_n320_etd2rk", steps=2)
    got, ref = run_pair(api, p)
    assert rel_err_inf(got, ref) <= TOL


def _paper_rows():
    from tests.test_oracle_paper import load_golden
    return [pytest.param(sizes, s, k, e, id=f"{'x'.join(map(str, sizes))}-{s}-{k}")
            for sizes, s, k, e in load_golden()]


@pytest.mark.parametrize("sizes,scheme,steps,err", _paper_rows())
def test_gpu_reproduces_paper_errors(api, sizes, scheme, steps, err):
    """The paper's own 3D ADR test (Section 4.2), every printed point (40x41x42 and
    80x81x82, exponential Euler, ETD2RK, Lawson-Euler, Lawson2b, up to 32800 steps):
    the CUDA path gives the relative error the paper prints
    (tests/golden/paper_adr_errors.txt) to 1e-8 of its value."""
    sch = {"etd2rk": wl.ETD2RK, "expeuler": wl.EXPEULER, "lawson_euler": wl.LAWSON_EULER,
           "lawson2b": wl.LAWSON2B}[scheme]
    p = wl.paper_adr_3d(sizes, steps, sch)
    plan, g, U = api.setup(p)
    api.expint_step(plan, sch, U, steps, g=g)
    e = rel_err_inf(U.cpu().numpy(), math.e * p.u0)
    assert abs(e - err) <= 1e-8 * err, (e, err)


def test_zero_steps_and_tau_zero(api):
    p = wl.adr_3d(seed=1, steps=0, sizes=(8, 9, 10))
    plan, g, U = api.setup(p)
    U0 = U.clone()
    api.expint_step(plan, wl.ETD2RK, U, 0, g=g)
    assert torch.equal(U, U0)
    # tau = 0: phi_l = I/l!, the split action is V/l! for every l (Theorem 1 at tau = 0)
    plan0 = api.Plan(p.A, 0.0, 2)
    V = dev(wl.random_tensor((10, 9, 8), 2))
    for ell in range(3):
        P = api.mumode_phi_apply(plan0, ell, V)
        assert torch.allclose(P, V / math.factorial(ell), rtol=0, atol=1e-15)


def test_nonfinite_raises_status_flag(api):
    p = wl.adr_3d(seed=1, steps=1, sizes=(8, 9, 10))
    p.u0 = p.u0.copy()
    p.u0[3, 4, 5] = np.nan
    plan, g, U = api.setup(p)
    api.expint_step(plan, wl.EXPEULER, U, 1, g=g)
    assert plan.status(reset=True) & api.STATUS_NONFINITE
    assert plan.status() == 0


def test_error_codes(api):
    p = wl.adr_3d(seed=1, steps=1, sizes=(8, 9, 10))
    plan, g, U = api.setup(p, ell_max=1)
    with pytest.raises(api.PhisplitError) as e:       # ETD2RK needs ell_max >= 2
        api.expint_step(plan, wl.ETD2RK, U, 1, g=g)
    assert e.value.code == -1
    small = torch.empty(4, dtype=torch.float64, device="cuda")
    with pytest.raises(api.PhisplitError) as e:
        api.expint_step(plan, wl.EXPEULER, U, 1, g=g, ws=small)
    assert e.value.code == -8
    with pytest.raises(api.PhisplitError) as e:
        api.mumode_phi_apply(plan, 3, U)
    assert e.value.code == -1
    with pytest.raises(api.PhisplitError) as e:        # V and P overlap
        api.mumode_phi_apply(plan, 0, U, P=U)
    assert e.value.code == -1


def test_graph_replay_equals_direct_launches_fp64(api):
    p = wl.adr_3d(seed=5, steps=3, scheme=wl.ETD2RK, sizes=(20, 17, 13))
    plan, g, U = api.setup(p, "fp64")
    for k in range(3):
        api.expint_step(plan, p.scheme, U, 1, t0=k * p.tau, g=g)
    plan2, g2, V = api.setup(p, "fp64")
    plan2.set_graphs(False)
    api.expint_step(plan2, p.scheme, V, 3, g=g2)
    torch.cuda.synchronize()
    assert torch.equal(U, V)


@pytest.mark.parametrize("scheme", [wl.EXPROSEULER, wl.ETD2RK])
def test_lq_riccati_matches_oracle(api, scheme):
    """The paper's LQ-control Riccati problem (Section 4.1, banded non-tridiagonal A)
    at nhat = 12 (144 x 144 matrices), 10 steps; exponential Rosenbrock-Euler forms
    phi_1 of its Jacobian on the GPU every step (eq. (21))."""
    p = wl.lq_riccati(12, 10, scheme, T=0.025 * 10 / 170)
    got, ref = run_pair(api, p)
    assert rel_err_fro(got, ref) <= TOL and rel_err_inf(got, ref) <= TOL


def test_rosenbrock_rejects_other_nonlinearities(api):
    p = wl.allen_cahn_2d(n=16, seed=1, steps=1, scheme=wl.EXPEULER)
    plan, g, U = api.setup(p, "fp64", ell_max=1)
    with pytest.raises(api.PhisplitError) as e:
        api.expint_step(plan, wl.EXPROSEULER, U, 1, g=g)
    assert e.value.code == -3


def test_expeuler_alternative_form_matches_oracle(api):
    p = wl.adr_3d(seed=5, steps=4, scheme=wl.EXPEULER_ALT, sizes=(20, 17, 13))
    got, ref = run_pair(api, p)
    assert rel_err_inf(got, ref) <= TOL


@pytest.fixture(scope="module")
def lq_ref():
    """The paper's LQ problem (nhat = 30) at T = 0.025 from the oracle: Richardson
    extrapolation of ETD2RK at 170 and 340 steps, plus the printed errors."""
    from tests.test_oracle_paper import lq_golden, lq_reference
    ref, _ = lq_reference(30, 170)
    return ref, {(s, n): e for (_, s, n, e) in lq_golden(30)}


@pytest.mark.parametrize("scheme,prec", [(wl.ETD2RK, "fp64"), (wl.EXPROSEULER, "fp64"),
                                         (wl.ETD2RK, "bf16x3")])
def test_lq_riccati_reproduces_printed_errors(api, lq_ref, scheme, prec):
    """GPU runs of the paper's LQ problem (Section 4.1, nhat = 30) at 30 steps land on
    the errors printed in Figure "riccati" (ETD2RK 1.7186e-4, exponential
    Rosenbrock-Euler 1.6105e-4) to 0.5 %; the BF16x3 form adds ~1e-7 to them."""
    ref, printed = lq_ref
    p = wl.lq_riccati(30, 30, scheme)
    plan, g, U = api.setup(p, prec)
    api.expint_step(plan, scheme, U, 30, g=g)
    torch.cuda.synchronize()
    assert plan.status() == 0
    e = rel_err_fro(U.cpu().numpy(), ref)
    key = ("etd2rk" if scheme == wl.ETD2RK else "exprosenbrock", 30)
    assert abs(e / printed[key] - 1) < 5e-3, (e, printed[key])



def test_checkpoint_resume_is_bit_identical_fp64(api):
    p = wl.paper_adr_3d((20, 21, 22), steps=6, scheme=wl.ETD2RK)
    plan, g, U = api.setup(p, "fp64")
    api.expint_step(plan, p.scheme, U, 6, g=g)
    plan2, g2, V = api.setup(p, "fp64")
    api.expint_step(plan2, p.scheme, V, 4, g=g2)
    saved = V.cpu().numpy().copy()
    plan2.close()
    plan3, g3, W = api.setup(p, "fp64")
    W.copy_(torch.from_numpy(saved))
    api.expint_step(plan3, p.scheme, W, 2, t0=4 * p.tau, g=g3)   # time-dependent g
    torch.cuda.synchronize()
    assert torch.equal(U, W)


@pytest.mark.parametrize("scheme", [wl.EXPEULER, wl.ETD2RK])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("bf16x3", 1e-6), ("tf32x3", 1e-6)])
def test_lq_order4_matches_oracle(api, scheme, prec, tol):
    """The LQ problem as an order-4 tensor (the remark closing Section 4.1): four
    directions of nhat x nhat matrices D1^T, D2^T, D1^T, D2^T, and G = C + U B U on the
    matrix view of the state, against the oracle's order-4 run."""
    p = wl.lq_riccati_order4(8, 12, scheme)
    plan, g, U = api.setup(p, prec)
    api.expint_step(plan, scheme, U, p.steps, g=g)
    torch.cuda.synchronize()
    assert plan.status() == 0
    ref = integrate(OracleProblem.from_problem(p), p.u0, scheme, p.steps)
    got = U.cpu().numpy()
    assert rel_err_fro(got, ref) <= tol and rel_err_inf(got, ref) <= tol


def test_lq_order4_nhat30_converges_to_the_lq_solution(api, lq_ref):
    """The order-4 form of the paper's LQ problem (nhat = 30: four 30 x 30 phi
    matrices per phi-function instead of two 900 x 900 ones), FP64 on the GPU, against
    the two-direction form's extrapolated solution: the GPU's errors at 30 and 65
    steps are the oracle's order-4 errors (about 2.3e-4 and 4.8e-5, the size of the
    two-direction form's printed 1.72e-4 and 3.53e-5) and fall at second order."""
    ref, printed = lq_ref
    errs, oracle_errs = [], []
    for m in (30, 65):
        p = wl.lq_riccati_order4(30, m, wl.ETD2RK)
        plan, g, U = api.setup(p, "fp64")
        api.expint_step(plan, wl.ETD2RK, U, m, g=g)
        torch.cuda.synchronize()
        assert plan.status() == 0
        errs.append(rel_err_fro(U.cpu().numpy().reshape(ref.shape), ref))
        orc = integrate(OracleProblem.from_problem(p), p.u0, wl.ETD2RK, m)
        oracle_errs.append(rel_err_fro(orc.reshape(ref.shape), ref))
    order = math.log(errs[0] / errs[1]) / math.log(65 / 30)
    assert 1.9 < order < 2.2, (errs, order)
    for e, o in zip(errs, oracle_errs):
        assert abs(e / o - 1) < 1e-4, (errs, oracle_errs)
    assert 0.5 < errs[0] / printed[("etd2rk", 30)] < 2, errs


def test_rosenbrock_needs_the_two_direction_form(api):
    p = wl.lq_riccati_order4(6, 4, wl.EXPROSEULER)
    plan, g, U = api.setup(p, "fp64")
    with pytest.raises(api.PhisplitError):
        api.expint_step(plan, wl.EXPROSEULER, U, 1, g=g)


@pytest.fixture(scope="module")
def lq40_ref():
    """The paper's LQ problem at nhat = 40 (n = 1600) at T = 0.025 from the oracle on
    the host cores: Richardson extrapolation of ETD2RK at 100 and 200 steps, plus the
    printed errors of Figure "riccati_40"."""
    from tests.test_oracle_paper import lq_golden, lq_reference
    ref, _ = lq_reference(40, 100)
    return ref, {(s, n): e for (_, s, n, e) in lq_golden(40)}


@pytest.mark.parametrize("scheme,prec,steps", [(wl.ETD2RK, "fp64", 30), (wl.ETD2RK, "fp64", 65),
                                               (wl.EXPROSEULER, "fp64", 30), (wl.ETD2RK, "bf16x3", 30),
                                               (wl.ETD2RK, "tf32x3", 65)])
def test_lq_riccati_nhat40_reproduces_printed_errors(api, lq40_ref, scheme, prec, steps):
    """GPU runs of the paper's LQ problem at nhat = 40 (Section 4.1, Table
    "riccati_order_40") land on the errors printed in Figure "riccati_40" (ETD2RK
    1.9744e-4 at 30 steps and 4.0443e-5 at 65, exponential Rosenbrock-Euler 1.7195e-4
    at 30) to 0.5 %."""
    ref, printed = lq40_ref
    p = wl.lq_riccati(40, steps, scheme)
    plan, g, U = api.setup(p, prec)
    api.expint_step(plan, scheme, U, steps, g=g)
    torch.cuda.synchronize()
    assert plan.status() == 0
    e = rel_err_fro(U.cpu().numpy(), ref)
    key = ("etd2rk" if scheme == wl.ETD2RK else "exprosenbrock", steps)
    assert abs(e / printed[key] - 1) < 5e-3, (e, printed[key])
