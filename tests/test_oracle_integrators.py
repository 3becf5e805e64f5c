"""Pins of the oracle's K u, g and time steppers (Section 2, Section 3.2).

Against: the assembled Kronecker sum (eq. (1b)), the Riccati vec form (eq. (3)),
exactness statements of Section 2 (exponential Euler exact for linear
constant-coefficient problems, Lawson-Euler exact for linear homogeneous ones),
and observed convergence orders against an independent high-accuracy ODE
solve (scipy.integrate.solve_ivp), as in the paper's order tables.
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

import oracle.integrators as oi
from oracle.integrators import OracleProblem, kron_apply, g_eval, integrate
from paper_2304_02327_gb300 import workloads as wl
from tests.test_oracle_tucker import kron_sum, vec


def test_kron_apply_equals_assembled_K():
    ns = (4, 3, 5)
    As = [wl.fd_matrix(n, 0.4, -0.9) + 0.2 * wl.random_dense(n, 10 + n) for n in ns]
    U = wl.random_tensor(tuple(reversed(ns)), 3)
    assert np.abs(vec(kron_apply(U, As)) - kron_sum(As) @ vec(U)).max() < 1e-12


def test_riccati_kronecker_form_eq3():
    n = 6
    p = wl.riccati_2d(n, seed=2)
    op = OracleProblem.from_problem(p, lmax=1)
    Um = np.random.default_rng(0).standard_normal((n, n))
    Ust = np.ascontiguousarray(Um.T)                         # stored (n_2, n_1)
    KU = kron_apply(Ust, p.A).T
    assert np.abs(KU - (p.A[0] @ Um + Um @ p.A[1].T)).max() < 1e-9
    # eq. (3): ((I (x) A1) + (A2 (x) I)) vec(U) + vec(C + U B U), vec stacks columns
    Kmat = np.kron(np.eye(n), p.A[0]) + np.kron(p.A[1], np.eye(n))
    rhs = Kmat @ Um.reshape(-1, order="F") + (p.C.T + Um @ p.B @ Um).reshape(-1, order="F")
    got = vec(kron_apply(Ust, p.A) + g_eval(op, Ust))
    assert np.abs(got - rhs).max() < 1e-9 * np.abs(rhs).max()


def test_expeuler_d1_linear_is_exact():
    """d = 1 (no splitting): exponential Euler is exact for u' = A u + c (Section 2)."""
    n, tau = 12, 0.03
    A = wl.fd_matrix(n, 0.2, 0.5)
    u = wl.random_tensor((n,), 1)
    c = 0.3
    op = OracleProblem(A=[A], tau=tau, g_kind=oi.G_CUBIC, cubic=(c, 0, 0, 0))
    got = integrate(op, u, oi.EXPEULER, 3)
    Z = np.zeros((n + 1, n + 1))
    Z[:n, :n] = A
    Z[:n, n] = c
    ref = (scipy.linalg.expm(3 * tau * Z) @ np.append(u, 1.0))[:n]
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("scheme", [oi.LAWSON_EULER, oi.LAWSON2B])
def test_lawson_linear_homogeneous_is_exact(scheme):
    """g = 0: Lawson schemes give e^{tau K} u per step, no splitting error (Section 3.2)."""
    ns = (4, 5)
    As = [wl.fd_matrix(n, 0.3, 0.4) for n in ns]
    U = wl.random_tensor(tuple(reversed(ns)), 2)
    op = OracleProblem(A=As, tau=0.05)
    got = integrate(op, U, scheme, 4)
    ref = scipy.linalg.expm(0.2 * kron_sum(As)) @ vec(U)
    assert np.abs(vec(got) - ref).max() < 1e-12


def small_adr(ns=(5, 6, 4), eps=0.05, beta=0.5, seed=8):
    As = [wl.fd_matrix(n, eps, beta) for n in ns]
    U0 = 0.5 + 0.3 * wl.random_tensor(tuple(reversed(ns)), seed)
    return As, U0


def reference_solution(As, U0, cubic, T):
    K = kron_sum(As)
    c0, c1, c2, c3 = cubic
    f = lambda t, u: K @ u + c0 + c1 * u + c2 * u * u + c3 * u * u * u
    sol = scipy.integrate.solve_ivp(f, (0, T), vec(U0), method="DOP853",
                                    rtol=1e-13, atol=1e-14)
    return sol.y[:, -1]


def observed_orders(scheme, cubic=(0.0, -0.5, 1.5, -1.0), T=0.5, steps=(8, 16, 32, 64)):
    As, U0 = small_adr()
    ref = reference_solution(As, U0, cubic, T)
    errs = []
    for m in steps:
        op = OracleProblem(A=As, tau=T / m, g_kind=oi.G_CUBIC, cubic=cubic)
        errs.append(np.abs(vec(integrate(op, U0, scheme, m)) - ref).max())
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


@pytest.mark.parametrize("scheme,order", [(oi.EXPEULER, 1), (oi.ETD2RK, 2),
                                          (oi.LAWSON_EULER, 1), (oi.LAWSON2B, 2),
                                          (oi.EXPEULER_ALT, 1)])
def test_observed_order(scheme, order):
    """Global order on a step sweep: 1 for (Lawson-/exponential) Euler, 2 for
    ETD2RK and Lawson2b, as in the paper's order tables (Section 4)."""
    o = observed_orders(scheme)
    assert abs(o[-1] - order) < 0.15, o


def test_planted_missing_factor_breaks_etd2rk_order(monkeypatch):
    """A planted mistake in the oracle -- dropping the (2!)^(d-1) factor of the
    phi_2 stage (eq. (20) as printed) -- must fail the order pin."""
    real = oi.phisplit_apply

    def wrong(V, phis, ell):
        out = real(V, phis, ell)
        return out / 2 ** (V.ndim - 1) if ell == 2 else out

    monkeypatch.setattr(oi, "phisplit_apply", wrong)
    o = observed_orders(oi.ETD2RK)
    assert abs(o[-1] - 2) > 0.5, o


def test_planted_missing_tau_breaks_consistency(monkeypatch):
    """Planting the other reading of eq. (20) (tau on G only) gives an
    inconsistent scheme: the error does not decrease with the step."""
    def wrong_step(op, U, scheme, t=0.0):
        Gn = g_eval(op, U, t)
        W1 = kron_apply(U, op.A) / op.tau + Gn
        U2 = U + op.tau * oi.phisplit_apply(W1, op.phi_list(1), 1)
        return U2 + op.tau * oi.phisplit_apply(g_eval(op, U2, t + op.tau) - Gn, op.phi_list(2), 2)

    monkeypatch.setattr(oi, "step", wrong_step)
    with np.errstate(all="ignore"):
        o = observed_orders(oi.ETD2RK, steps=(8, 16, 32))
    # either it diverges (nan/inf) or the error stops decreasing
    assert not (abs(o[-1] - 2) < 0.5), o


def riccati_small(n1=6, n2=5, seed=3):
    rng = np.random.default_rng(seed)
    A = [wl.fd_matrix(n1, 0.3, 0.4), wl.fd_matrix(n2, 0.2, -0.3)]
    B = 0.3 * rng.standard_normal((n2, n1))
    C = 0.5 * rng.standard_normal((n2, n1))          # stored like U: (n2, n1)
    U0 = 0.2 * rng.standard_normal((n2, n1))
    return A, B, C, U0


def riccati_rhs_vec(A, B, C, n1, n2):
    """u' for the column-stacked matrix U (n1 x n2): A1 U + U A2^T + C + U B U."""
    Cm = C.T

    def f(t, u):
        Um = u.reshape(n2, n1).T
        return (A[0] @ Um + Um @ A[1].T + Cm + Um @ B @ Um).T.reshape(-1)
    return f


def test_riccati_jacobian_is_the_linearisation():
    """K + dG(U) = J_2 (+) J_1: the Kronecker sum of the oracle's J matches a
    finite-difference Jacobian of the Riccati right-hand side (Section 4.1)."""
    n1, n2 = 6, 5
    A, B, C, U0 = riccati_small(n1, n2)
    op = OracleProblem(A=A, tau=0.1, g_kind=oi.G_RICCATI, B=B, C=C)
    J = oi.riccati_jacobian(op, U0)
    f = riccati_rhs_vec(A, B, C, n1, n2)
    u0 = U0.reshape(-1)
    h = 1e-6
    fd = np.stack([(f(0, u0 + h * e) - f(0, u0 - h * e)) / (2 * h) for e in np.eye(n1 * n2)], axis=1)
    assert np.abs(kron_sum(J) - fd).max() < 1e-7 * max(1.0, np.abs(fd).max())


def test_rosenbrock_linear_problem_is_exponential_euler():
    """B = 0: the Jacobian is K itself, so exponential Rosenbrock-Euler is exponential
    Euler (eq. (13) with K_n = K), step for step."""
    A, B, C, U0 = riccati_small()
    op = OracleProblem(A=A, tau=0.05, g_kind=oi.G_RICCATI, B=0.0 * B, C=C)
    op.ensure_phis(1)
    a = oi.step(op, U0, oi.EXPROSEULER)
    b = oi.step(op, U0, oi.EXPEULER)
    assert np.abs(a - b).max() < 1e-14 * np.abs(b).max()


def test_rosenbrock_observed_order_two():
    """Exponential Rosenbrock-Euler (PHISPLIT) on a small Riccati problem: global order 2
    on a step sweep against scipy's DOP853 on the assembled system, as the paper's
    order table for the LQ problem shows (Section 4.1)."""
    n1, n2 = 6, 5
    A, B, C, U0 = riccati_small(n1, n2)
    T = 0.4
    f = riccati_rhs_vec(A, B, C, n1, n2)
    ref = scipy.integrate.solve_ivp(f, (0, T), U0.reshape(-1), method="DOP853", rtol=1e-13,
                                    atol=1e-14).y[:, -1]
    errs = []
    for m in (8, 16, 32, 64):
        op = OracleProblem(A=A, tau=T / m, g_kind=oi.G_RICCATI, B=B, C=C)
        errs.append(np.abs(integrate(op, U0, oi.EXPROSEULER, m).reshape(-1) - ref).max())
    o = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert abs(o[-1] - 2) < 0.15, o


def test_lq_riccati_reaches_the_algebraic_riccati_solution():
    """The paper's LQ problem (Section 4.1) at a small grid: both second-order schemes
    run to the steady state, the solution of A^T U + U A + C + U B U = 0, which scipy's
    continuous algebraic Riccati solver gives independently (B = -b b^T, C = alpha c^T c)."""
    nhat, T, steps = 6, 0.5, 100
    p = wl.lq_riccati(nhat, steps, wl.ETD2RK, T=T)
    A = p.A[0].T                                        # the system matrix
    xi = np.tile(wl.grid(nhat), nhat)
    b = ((xi > 0.1) & (xi <= 0.3)).astype(float)[:, None]
    Cm = p.C.T
    X = scipy.linalg.solve_continuous_are(A, b, Cm, np.eye(1))
    for scheme in (oi.ETD2RK, oi.EXPROSEULER):
        op = OracleProblem.from_problem(p, lmax=2)
        U = integrate(op, p.u0, scheme, steps)
        assert oi.rel_err_fro(U.T, X) < 1e-6, scheme


def test_expeuler_alternative_form_exact_for_linear_problems():
    """The alternative exponential Euler form (Section 3.2) is exact for linear
    autonomous problems: with g = 0 it is e^{tau K} u, step after step."""
    ns = (4, 5, 3)
    As = [wl.fd_matrix(n, 0.3, 0.2) for n in ns]
    U = wl.random_tensor(tuple(reversed(ns)), 2)
    op = OracleProblem(A=As, tau=0.07)
    got = integrate(op, U, oi.EXPEULER_ALT, 3)
    ref = scipy.linalg.expm(0.21 * kron_sum(As)) @ vec(U)
    assert np.abs(vec(got) - ref).max() < 1e-12


@pytest.mark.parametrize("scheme", [oi.EXPEULER, oi.ETD2RK, oi.LAWSON_EULER])
@pytest.mark.parametrize("kind", ["adr", "riccati"])
def test_step_at_is_the_sampled_full_step(scheme, kind):
    """step_at (one step restricted to a sampled output grid, used on states too large
    to step in full) equals the full step on that grid, for tensors and for the
    Riccati form, including sets that skip, repeat no index and end at the edge."""
    if kind == "adr":
        p = wl.adr_3d(seed=3, sizes=(9, 7, 6), tau=2e-3)
        sets = [np.array([0, 3, 8]), np.array([1, 6]), np.array([0, 2, 5])]
    else:
        p = wl.riccati_2d(10, seed=4, tau=1e-3)
        p.u0 = 0.1 * wl.random_tensor((10, 10), 5)
        sets = [np.array([0, 4, 9]), np.array([2, 3, 7, 9])]
    op = OracleProblem.from_problem(p)
    U = np.asarray(p.u0, dtype=np.float64)
    full = oi.step(op, U, scheme, 0.25)
    got = oi.step_at(op, U, scheme, 0.25, sets)
    ref = full[np.ix_(*reversed(sets))]
    assert got.shape == ref.shape
    assert np.abs(got - ref).max() <= 1e-14 * np.abs(full).max()


def _lq_pair(nhat, steps, scheme):
    p2 = wl.lq_riccati(nhat, steps, scheme)
    p4 = wl.lq_riccati_order4(nhat, steps, scheme)
    return p2, p4, OracleProblem.from_problem(p2), OracleProblem.from_problem(p4)


def test_lq_order4_operator_is_the_two_direction_operator():
    """The remark closing Section 4.1: A^T U + U A of the LQ problem is the order-4
    Kronecker sum of D1^T, D2^T, D1^T, D2^T on the same memory, and G = C + U B U
    is the same function of the state in both forms."""
    nhat = 5
    p2, p4, op2, op4 = _lq_pair(nhat, 10, oi.ETD2RK)
    U2 = 0.1 * wl.random_tensor((nhat * nhat, nhat * nhat), 3)
    U4 = U2.reshape((nhat,) * 4)
    K2, K4 = kron_apply(U2, p2.A), kron_apply(U4, p4.A)
    assert np.abs(K4.reshape(U2.shape) - K2).max() <= 1e-12 * np.abs(K2).max()
    G2, G4 = g_eval(op2, U2), g_eval(op4, U4)
    assert np.abs(G4.reshape(U2.shape) - G2).max() <= 1e-14 * np.abs(G2).max()


def test_lq_order4_lawson_step_equals_two_direction_form():
    """For l = 0 the direction split is exact (eq. (5)-(6)): a Lawson-Euler step of the
    order-4 form (four 6 x 6 exponentials) equals that of the two-direction form
    (two 36 x 36 exponentials)."""
    nhat = 6
    p2, p4, op2, op4 = _lq_pair(nhat, 20, oi.LAWSON_EULER)
    U2 = 0.05 * wl.random_tensor((nhat * nhat, nhat * nhat), 4)
    a = oi.step(op2, U2, oi.LAWSON_EULER)
    b = oi.step(op4, U2.reshape((nhat,) * 4), oi.LAWSON_EULER).reshape(U2.shape)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_lq_order4_etd2rk_converges_at_order_two_to_the_same_solution():
    """The order-4 form splits phi_1, phi_2 over four directions instead of two, so
    its ETD2RK differs from the two-direction form's by O(tau^2) per unit time; both
    converge at order two to the same solution (a fine two-direction run here)."""
    nhat = 6
    p, _, op, _ = _lq_pair(nhat, 400, oi.ETD2RK)
    ref = integrate(op, p.u0, oi.ETD2RK, 400)
    errs = []
    for m in (10, 20, 40):
        p4 = wl.lq_riccati_order4(nhat, m, oi.ETD2RK)
        got = integrate(OracleProblem.from_problem(p4), p4.u0, oi.ETD2RK, m)
        errs.append(oi.rel_err_fro(got.reshape(ref.shape), ref))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 < o < 2.3 for o in orders), (errs, orders)
