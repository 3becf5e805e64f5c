"""Parity of the split-precision tensor-core forms (tcgen05) with the FP64 oracle.

Both mixed forms are run by every test: TF32x3 (operand in two TF32 parts,
Phi in three) and BF16x3 (operand and Phi in three BF16 parts each).

Tolerances come from the arithmetic: operands are split x = hi + lo with
|x - hi - lo| <= 2^-24 |x|, products drop lo*lo (<= 2^-22 |ab| relative to the
TF32 grid), sums accumulate in FP32 over K <= 320 terms and intermediates are
stored in FP32.  One mu-mode product is therefore accurate to a few 2^-24 of
sum_j |Phi_ij||V_j|; for the smooth/decaying phi matrices here that stays below
2e-6 of max|P| for a whole Tucker chain (d <= 4).  Integrations add the FP64
update U + tau Y, so their error relative to max|U| is far smaller; the stated
tolerance of the mixed form is 1e-6 relative in the infinity norm.
"""
import numpy as np
import pytest
import torch

from oracle.integrators import OracleProblem, g_eval, integrate, kron_apply, rel_err_inf, rel_err_fro
from oracle.phi import phi_matrices
from oracle.tucker import phisplit_apply, phisplit_apply_at
from paper_2304_02327_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL_APPLY = 4e-6
TOL_STEP = 1e-6
# Lawson schemes pass the whole state through the Tucker operator every step, so
# the contraction's relative error (measured: a one-sided bias of about
# 2e-7 (n/128) per mode, from the tensor core truncating toward zero) lands on U
# directly instead of on the increment tau*Y: 5e-7 per step is stated for them.
TOL_LAWSON_PER_STEP = 5e-7


FORMS = ["tf32x3", "bf16x3"]


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2304_02327_gb300 import api as _api, build
    build.build()
    _api.lib()
    return _api


@pytest.fixture(params=FORMS)
def form(request):
    return request.param


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


@pytest.mark.parametrize("ns", [(64,), (128, 128), (33, 17), (48, 64, 80), (320, 40, 2),
                                (20, 17, 13), (5, 4, 3, 6), (128, 300), (1, 9, 4), (127, 3),
                                (3, 127, 1)])
@pytest.mark.parametrize("ell", [0, 1, 2])
def test_mixed_mumode_apply_matches_oracle(api, form, ns, ell):
    tau = 2e-3
    As = [wl.fd_matrix(n, 0.4, 0.9) for n in ns]
    V = wl.random_tensor(tuple(reversed(ns)), seed=len(ns) * 11 + ell)
    plan = api.Plan(As, tau, 2, form)
    P = api.mumode_phi_apply(plan, ell, dev(V), alpha=1.0)
    torch.cuda.synchronize()
    assert plan.status() == 0
    ref = phisplit_apply(V, [phi_matrices(tau * A, 2)[ell] for A in As], ell)
    assert rel_err_inf(P.cpu().numpy(), ref) <= TOL_APPLY


def test_mixed_dense_random_operator(api, form):
    """Dense, non-decaying matrices: error measured against sum |Phi| |V| bounds."""
    ns = (96, 80)
    As = [0.3 * wl.random_dense(n, 3 + n) for n in ns]
    V = wl.random_tensor((80, 96), 5)
    plan = api.Plan(As, 1.0, 1, form)
    P = api.mumode_phi_apply(plan, 1, dev(V)).cpu().numpy()
    phis = [phi_matrices(A, 1)[1] for A in As]
    ref = phisplit_apply(V, phis, 1)
    bound = phisplit_apply(np.abs(V), [np.abs(m) for m in phis], 1)
    assert np.max(np.abs(P - ref) / bound) <= 64 * 2.0**-24


def run_pair(api, p, prec):
    plan, g, U = api.setup(p, prec)
    api.expint_step(plan, p.scheme, U, p.steps, g=g)
    torch.cuda.synchronize()
    assert plan.status() == 0
    ref = integrate(OracleProblem.from_problem(p), p.u0, p.scheme, p.steps)
    return U.cpu().numpy(), ref


@pytest.mark.parametrize("scheme", [wl.EXPEULER, wl.ETD2RK, wl.LAWSON_EULER, wl.LAWSON2B])
def test_mixed_schemes_small(api, form, scheme):
    p = wl.adr_3d(seed=5, steps=5, scheme=scheme, sizes=(40, 33, 24))
    got, ref = run_pair(api, p, form)
    lawson = scheme in (wl.LAWSON_EULER, wl.LAWSON2B)
    assert rel_err_inf(got, ref) <= (TOL_LAWSON_PER_STEP * p.steps if lawson else TOL_STEP)


def test_mixed_allen_cahn_n64(api, form):
    p = wl.workload("ac2d_n64_expeuler")
    got, ref = run_pair(api, p, form)
    assert rel_err_inf(got, ref) <= TOL_STEP


def test_mixed_adr3d_n128_full(api, form):
    """3D ADR n = 128, 100 ETD2RK steps in the mixed form against the FP64 oracle."""
    p = wl.workload("adr3d_n128_etd2rk")
    got, ref = run_pair(api, p, form)
    assert rel_err_inf(got, ref) <= TOL_STEP and rel_err_fro(got, ref) <= TOL_STEP


def test_mixed_adr3d_n320_two_steps(api, form):
    """3D ADR at n = 320 (N = 32.8M), two ETD2RK steps, mixed form vs the FP64 oracle."""
    p = wl.workload("adr3d_n320_etd2rk", steps=2)
    got, ref = run_pair(api, p, form)
    assert rel_err_inf(got, ref) <= TOL_STEP


def test_mixed_paper_adr_error(api, form):
    """The paper's ADR test at 40x41x42, 40 ETD2RK steps: the mixed form reproduces the
    printed error 3.034138277914e-4 to the mixed tolerance."""
    p = wl.paper_adr_3d((40, 41, 42), 40, wl.ETD2RK)
    plan, g, U = api.setup(p, form)
    api.expint_step(plan, wl.ETD2RK, U, 40, g=g)
    e = rel_err_inf(U.cpu().numpy(), np.e * p.u0)
    assert abs(e - 0.0003034138277914) <= 1e-6, e


def test_mixed_direction_600(api, form):
    """n = 600 (beyond one CTA's 128 output columns many times over, K = 600 in 19/10
    K-blocks), both modes, against the oracle."""
    As = [wl.fd_matrix(600, 0.1, 0.3), wl.fd_matrix(40, 0.2)]
    V = wl.random_tensor((40, 600), 21)
    plan = api.Plan(As, 1e-3, 1, form)
    P = api.mumode_phi_apply(plan, 1, dev(V)).cpu().numpy()
    ref = phisplit_apply(V, [phi_matrices(1e-3 * A, 1)[1] for A in As], 1)
    assert rel_err_inf(P, ref) <= TOL_APPLY


def test_mixed_large_direction_split_across_ctas(api, form):
    """n = 400 runs with its output columns split over several CTAs."""
    As = [wl.fd_matrix(400, 0.3, 0.5), wl.fd_matrix(24, 0.2)]
    V = wl.random_tensor((24, 400), 9)
    plan = api.Plan(As, 1e-3, 1, form)
    P = api.mumode_phi_apply(plan, 1, dev(V)).cpu().numpy()
    ref = phisplit_apply(V, [phi_matrices(1e-3 * A, 1)[1] for A in As], 1)
    assert rel_err_inf(P, ref) <= TOL_APPLY


# A dense remainder R_mu = A_mu - band that is not small puts the operand split's
# own rounding on K u: TF32x3 keeps the tensor operand to 2^-22 (two TF32 parts),
# BF16x3 to ~2^-25 (three BF16 parts), relative to sum |R||U| per product.  For
# the O(1) random remainder below that is 2^-22 * (sum|R||U| / |K u|, about 4 here)
# on the increment of each step: 2e-6 is stated for TF32x3 on it, 1e-6 for BF16x3.
TOL_DENSE_REMAINDER = {"tf32x3": 2e-6, "bf16x3": 1e-6}


def test_mixed_dense_operator_cubic(api, form):
    """Non-tridiagonal A_mu (d = 2): band stencil plus the remainder products
    R1 U + U R2^T on the tensor cores, cubic g, ETD2RK."""
    ns = (96, 80)
    As = [wl.fd_matrix(n, 0.3, 0.2) + 0.3 * wl.random_dense(n, 7 + n) for n in ns]
    p = wl.Problem(name="dense", A=As, u0=wl.random_tensor((80, 96), 3), g_kind=wl.G_CUBIC,
                   cubic=(0.1, 1.0, 0.0, -1.0), tau=1e-2, steps=3, scheme=wl.ETD2RK)
    got, ref = run_pair(api, p, form)
    assert rel_err_inf(got, ref) <= TOL_DENSE_REMAINDER[form]


@pytest.mark.parametrize("scheme", [wl.EXPEULER, wl.ETD2RK])
def test_mixed_riccati_matches_oracle(api, form, scheme):
    """Matrix Riccati (A = h^-2 tridiag(1,-2,1) + 0.1 skew, G = C + U B U, U0 = 0) in
    the mixed form: every product on the tensor cores except the band stencil."""
    p = wl.riccati_2d(192, seed=9, tau=1e-4, steps=10, scheme=scheme)
    got, ref = run_pair(api, p, form)
    assert rel_err_fro(got, ref) <= TOL_STEP and rel_err_inf(got, ref) <= TOL_STEP


def test_mixed_riccati_nonsquare_nonzero_start(api, form):
    """n1 != n2 (B is n2 x n1), a smooth nonzero U0 so that U B U matters from the
    first step (rough data would decay by orders of magnitude within a few steps and
    leave a relative error measured against a much smaller final state)."""
    n1, n2 = 96, 136
    rng = np.random.default_rng(12)
    A = [wl.fd_matrix(n, 1.0) + 0.1 * (lambda G: (G - G.T) / np.sqrt(2))(rng.standard_normal((n, n)))
         for n in (n1, n2)]
    B = 0.1 * rng.standard_normal((n2, n1))
    C = 0.01 * rng.standard_normal((n2, n1))
    x1, x2 = wl.grid(n1), wl.grid(n2)
    u0 = 0.5 * np.sin(2 * np.pi * x2)[:, None] * np.sin(np.pi * x1)[None, :]
    p = wl.Problem(name="riccati_ns", A=A, u0=u0, g_kind=wl.G_RICCATI, B=B, C=C, tau=1e-4,
                   steps=6, scheme=wl.ETD2RK)
    got, ref = run_pair(api, p, form)
    assert rel_err_fro(got, ref) <= TOL_STEP and rel_err_inf(got, ref) <= TOL_STEP


def test_mixed_riccati_n2048_sampled_last_step(api, form):
    """Riccati at full size (n = 2048, tau = 1e-4, exponential Euler, U0 = 0): after
    49 steps of the mixed form, the 50th is compared with the oracle's step from the
    same FP64 state on a 64 x 64 grid of sampled entries.  The oracle forms
    W = K U + G(U) in full and the Tucker only on the sampled rows of phi_1."""
    p = wl.workload("riccati_n2048_expeuler")
    plan, g, U = api.setup(p, form)
    api.expint_step(plan, p.scheme, U, p.steps - 1, g=g)
    Un = U.cpu().numpy()
    api.expint_step(plan, p.scheme, U, 1, g=g, t0=(p.steps - 1) * p.tau)
    got = U.cpu().numpy()
    assert plan.status() == 0
    op = OracleProblem.from_problem(p, lmax=1)
    W = kron_apply(Un, op.A) + g_eval(op, Un)
    rng = np.random.default_rng(77)
    I1 = np.sort(rng.choice(2048, 64, replace=False))
    I2 = np.sort(rng.choice(2048, 64, replace=False))
    ref = Un[np.ix_(I2, I1)] + p.tau * phisplit_apply_at(W, op.phi_list(1), 1, [I1, I2])
    err = np.max(np.abs(got[np.ix_(I2, I1)] - ref)) / np.max(np.abs(ref))
    # The stiff modes damp what earlier steps got wrong (the whole 50-step run lands
    # at 3.5e-7), so a single step is held to a tenth of the run's tolerance.
    assert err <= TOL_STEP / 10, err


def test_graph_replay_equals_direct_launches(api, form):
    """expint_step replays a captured graph by default; repeated calls (and calls on a
    second state with the same plan, which need their own graph) must give exactly the
    results of direct launches."""
    p = wl.adr_3d(seed=5, steps=4, scheme=wl.ETD2RK, sizes=(40, 33, 24))
    plan, g, U = api.setup(p, form)
    U2 = U.clone()
    ws = api.expint_workspace(plan, p.scheme, g)
    for k in range(4):                       # one capture, three replays
        api.expint_step(plan, p.scheme, U, 1, t0=k * p.tau, g=g, ws=ws)
    api.expint_step(plan, p.scheme, U2, 2, g=g, ws=ws)   # another key: nsteps, state
    api.expint_step(plan, p.scheme, U2, 2, t0=2 * p.tau, g=g, ws=ws)
    torch.cuda.synchronize()
    plan2, g2, V = api.setup(p, form)
    plan2.set_graphs(False)
    api.expint_step(plan2, p.scheme, V, 4, g=g2)
    torch.cuda.synchronize()
    assert torch.equal(U, V) and torch.equal(U2, V)



def test_checkpoint_resume_is_bit_identical(api, form):
    """A one-step method's state is (U_n, t_n): saving U after 3 of 6 steps, destroying
    the plan, rebuilding it from (A_mu, tau) and continuing gives exactly the
    uninterrupted run."""
    p = wl.adr_3d(seed=5, steps=6, scheme=wl.ETD2RK, sizes=(40, 33, 24))
    plan, g, U = api.setup(p, form)
    api.expint_step(plan, p.scheme, U, 6, g=g)
    plan2, g2, V = api.setup(p, form)
    api.expint_step(plan2, p.scheme, V, 3, g=g2)
    saved = V.cpu().numpy().copy()
    plan2.close()
    del V
    plan3, g3, W = api.setup(p, form)
    W.copy_(torch.from_numpy(saved))
    api.expint_step(plan3, p.scheme, W, 3, t0=3 * p.tau, g=g3)
    torch.cuda.synchronize()
    assert torch.equal(U, W)


@pytest.mark.parametrize("sizes", [(33, 20, 12), (40, 33, 24)])
def test_mixed_3d_prepass_both_marches(api, form, sizes):
    """The 3D K u + g prepass runs TMA-fed when the first direction is even (the FP64
    rows are then 16-byte multiples) and register-fed otherwise: both against the
    oracle, ETD2RK."""
    p = wl.adr_3d(seed=8, steps=4, scheme=wl.ETD2RK, sizes=sizes)
    got, ref = run_pair(api, p, form)
    assert rel_err_inf(got, ref) <= TOL_STEP and rel_err_fro(got, ref) <= TOL_STEP


@pytest.mark.parametrize("sizes", [(2, 3, 5), (64, 1, 7), (1, 40, 3), (34, 33, 1)])
def test_mixed_thin_3d_grids(api, form, sizes):
    """Degenerate 3D grids (a direction of size 1 or 2, tiles far wider than the grid,
    the zero-filled halo on every side) through both prepass marches and the
    contraction, ETD2RK, against the oracle."""
    p = wl.adr_3d(seed=9, steps=3, scheme=wl.ETD2RK, sizes=sizes)
    got, ref = run_pair(api, p, form)
    assert rel_err_inf(got, ref) <= TOL_STEP and rel_err_fro(got, ref) <= TOL_STEP


@pytest.mark.parametrize("scheme", [wl.EXPEULER, wl.ETD2RK])
def test_mixed_nonfinite_state_raises_status(api, form, scheme):
    """A NaN planted on the host in the initial state reaches the plan's status word
    through the split-precision update passes."""
    p = wl.adr_3d(seed=5, steps=2, scheme=scheme, sizes=(40, 33, 24))
    p.u0[3, 4, 5] = np.nan
    plan, g, U = api.setup(p, form)
    api.expint_step(plan, p.scheme, U, 2, g=g)
    torch.cuda.synchronize()
    assert plan.status(reset=True) & api.STATUS_NONFINITE
    assert plan.status() == 0
