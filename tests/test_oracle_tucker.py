"""Pins of the oracle's mu-mode product, Tucker operator and PHISPLIT action.

Against: the Kronecker-matrix form (eq. (5)), the element loop (eq. (7)), the
2D matrix form e^{A_1} V (e^{A_2})^T (Section 1), the exact e^{tau K} v of a
Kronecker sum (eq. (1b), scipy.linalg.expm), Theorem 1 (eq. (14)) and its
scalar special case.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg

from oracle.phi import phi_matrices
from oracle.tucker import mode_product, tucker, phisplit_apply, phisplit_apply_at
from paper_2304_02327_gb300 import workloads as wl


def vec(T):
    """Column-stacking vec of a tensor stored as (n_d, ..., n_1): i_1 fastest."""
    return np.asarray(T).reshape(-1)


def kron_chain(Ms):
    """M_d (x) ... (x) M_1 (eq. (5))."""
    K = np.ones((1, 1))
    for M in reversed(Ms):
        K = np.kron(K, M)
    return K


def kron_sum(As):
    """A_d (+) ... (+) A_1 = sum_mu I_d (x) .. (x) A_mu (x) .. (x) I_1 (eq. (1b))."""
    ns = [A.shape[0] for A in As]
    N = int(np.prod(ns))
    K = np.zeros((N, N))
    for mu in range(len(As)):
        Ms = [np.eye(n) for n in ns]
        Ms[mu] = As[mu]
        K += kron_chain(Ms)
    return K


@pytest.mark.parametrize("ns", [(3,), (2, 3), (3, 2), (2, 3, 4), (4, 1, 3), (3, 2, 2, 2)])
def test_tucker_equals_kronecker_matrix(ns):
    rng = np.random.default_rng(sum(ns))
    Ms = [rng.standard_normal((n, n)) for n in ns]
    V = rng.standard_normal(tuple(reversed(ns)))
    Y = tucker(V, Ms)
    ref = kron_chain(Ms) @ vec(V)
    assert np.abs(vec(Y) - ref).max() < 1e-13 * np.abs(ref).max()


def test_tucker_equals_element_loop_eq7():
    ns = (3, 4, 2)
    rng = np.random.default_rng(5)
    Ms = [rng.standard_normal((n, n)) for n in ns]
    V = rng.standard_normal(tuple(reversed(ns)))
    Y = tucker(V, Ms)
    for i1, i2, i3 in itertools.product(*(range(n) for n in ns)):
        s = 0.0
        for j1, j2, j3 in itertools.product(*(range(n) for n in ns)):
            s += V[j3, j2, j1] * Ms[0][i1, j1] * Ms[1][i2, j2] * Ms[2][i3, j3]
        assert abs(Y[i3, i2, i1] - s) < 1e-13


def test_two_dim_is_left_right_product():
    # V x_1 M1 x_2 M2 = M1 V M2^T for the n1 x n2 matrix V (Section 1)
    rng = np.random.default_rng(6)
    n1, n2 = 5, 7
    M1, M2 = rng.standard_normal((n1, n1)), rng.standard_normal((n2, n2))
    Vm = rng.standard_normal((n1, n2))
    Y = tucker(np.ascontiguousarray(Vm.T), [M1, M2])      # stored (n2, n1)
    assert np.abs(Y.T - M1 @ Vm @ M2.T).max() < 1e-13


def test_mode_product_single_direction():
    rng = np.random.default_rng(7)
    V = rng.standard_normal((4, 3, 5))   # n1=5, n2=3, n3=4
    M = rng.standard_normal((3, 3))
    Y = mode_product(V, M, 2)
    for a in range(4):
        for c in range(5):
            assert np.abs(Y[a, :, c] - M @ V[a, :, c]).max() < 1e-14


@pytest.mark.parametrize("ns,tau", [((4, 5), 0.05), ((3, 4, 5), 0.02)])
def test_ell0_is_exact_exponential(ns, tau):
    """l = 0: the Tucker of e^{tau A_mu} equals e^{tau K} v exactly (eq. (5)-(6))."""
    As = [wl.fd_matrix(n, 0.3, 0.7) + 0.1 * wl.random_dense(n, n) for n in ns]
    rng = np.random.default_rng(1)
    V = rng.standard_normal(tuple(reversed(ns)))
    phis = [phi_matrices(tau * A, 0)[0] for A in As]
    P = phisplit_apply(V, phis, 0)
    ref = scipy.linalg.expm(tau * kron_sum(As)) @ vec(V)
    assert np.abs(vec(P) - ref).max() < 1e-12 * np.abs(ref).max()


def exact_phi_action(K, v, ell):
    """phi_l(K) v from scipy's expm of [[K, I, 0],[0, 0, I],[0, 0, 0]] (eq. (4b))."""
    N = K.shape[0]
    Z = np.zeros(((ell + 1) * N, (ell + 1) * N))
    Z[:N, :N] = K
    for b in range(ell):
        Z[b * N:(b + 1) * N, (b + 1) * N:(b + 2) * N] = np.eye(N)
    E = scipy.linalg.expm(Z)
    return E[:N, ell * N:(ell + 1) * N] @ v


@pytest.mark.parametrize("ell", [1, 2])
@pytest.mark.parametrize("d", [2, 3])
def test_theorem1_split_error_is_second_order(ell, d):
    """||phi_l(tau K) v - p_l^(2)|| = O(tau^2)  (Theorem 1, eq. (14))."""
    ns = [4, 5, 3][:d]
    As = [wl.fd_matrix(n, 1.0, 2.0) for n in ns]
    K = kron_sum(As)
    rng = np.random.default_rng(3)
    V = rng.standard_normal(tuple(reversed(ns)))
    errs = []
    taus = [1e-3 * 2.0**-k for k in range(4)]
    for tau in taus:
        p = vec(phisplit_apply(V, [phi_matrices(tau * A, ell)[ell] for A in As], ell))
        ex = exact_phi_action(tau * K, vec(V), ell)
        errs.append(np.abs(p - ex).max())
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(abs(s - 2.0) < 0.15 for s in slopes), slopes


@pytest.mark.parametrize("ell", [0, 1, 2, 3])
def test_scalar_case_is_product_of_scalar_phis(ell):
    """A_mu = a_mu I: output = (l!)^(d-1) prod_mu phi_l(tau a_mu) v exactly."""
    from tests.test_oracle_phi import scalar_phi
    a = [-3.0, 0.5, -20.0]
    ns = [3, 4, 2]
    tau = 0.1
    V = np.random.default_rng(4).standard_normal(tuple(reversed(ns)))
    P = phisplit_apply(V, [phi_matrices(tau * ai * np.eye(n), ell)[ell] for ai, n in zip(a, ns)], ell)
    f = math.factorial(ell) ** 2 * np.prod([scalar_phi(tau * ai, ell) for ai in a])
    assert np.abs(P - f * V).max() < 1e-14 * max(1, abs(f))


def test_theorem1_second_order_term_d2():
    """d = 2, l = 1, A_mu = a_mu I: split - exact = -tau^2 a_1 a_2 / 12 + O(tau^3)."""
    from tests.test_oracle_phi import scalar_phi
    a1, a2 = -2.0, 3.0
    for tau in (1e-2, 5e-3):
        split = phisplit_apply(np.ones((1, 1)), [phi_matrices(tau * a1 * np.eye(1), 1)[1],
                                                 phi_matrices(tau * a2 * np.eye(1), 1)[1]], 1)[0, 0]
        exact = scalar_phi(tau * (a1 + a2), 1)
        lead = -tau**2 * a1 * a2 / 12
        assert abs((split - exact) - lead) < 5 * tau**3 * abs(a1 * a2) * max(abs(a1), abs(a2))


@pytest.mark.parametrize("ell", [1, 2])
def test_split_at_tau_zero_is_phi_of_zero(ell):
    # (l!)^(d-1) (1/l!)^d = 1/l! = phi_l(0)  (Theorem 1 proof, Section 3)
    V = np.random.default_rng(9).standard_normal((3, 4, 5))
    P = phisplit_apply(V, [phi_matrices(np.zeros((n, n)), ell)[ell] for n in (5, 4, 3)], ell)
    assert np.abs(P - V / math.factorial(ell)).max() < 1e-15


def test_phisplit_at_sampled_entries_element_loop():
    """phisplit_apply_at on a sampled index grid equals the element loop of eq. (7)
    with the (l!)^(d-1) factor, entry by entry (brute force, d = 3, l = 2)."""
    rng = np.random.default_rng(31)
    ns = (5, 4, 6)
    phis = [rng.standard_normal((n, n)) for n in ns]
    V = rng.standard_normal(tuple(reversed(ns)))
    sets = [[4, 0, 2], [3], [1, 5]]
    got = phisplit_apply_at(V, phis, 2, sets)
    assert got.shape == (2, 1, 3)
    for a3, i3 in enumerate(sets[2]):
        for a2, i2 in enumerate(sets[1]):
            for a1, i1 in enumerate(sets[0]):
                acc = 0.0
                for j3, j2, j1 in itertools.product(range(ns[2]), range(ns[1]), range(ns[0])):
                    acc += phis[0][i1, j1] * phis[1][i2, j2] * phis[2][i3, j3] * V[j3, j2, j1]
                assert abs(4.0 * acc - got[a3, a2, a1]) <= 1e-12 * max(1.0, abs(acc))
