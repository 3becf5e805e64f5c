"""Pins of the oracle's e^X and phi_l(X) (Section 1 eq. (4a)-(4b), Section 3.1).

Each test fixes the oracle against something other than itself: an independent
library routine (scipy.linalg.expm), closed forms, the paper's own identities.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle.phi import expm_pade13, phi_matrices, pade_coefficients
from paper_2304_02327_gb300 import workloads as wl


def scalar_phi(z: float, ell: int) -> float:
    """phi_l(z) for a scalar: series for |z| < 1, else the recurrence
    phi_l(z) = (phi_{l-1}(z) - 1/(l-1)!)/z started from e^z (eq. (4a)-(4b))."""
    if abs(z) < 1.0:
        return sum(z**i / math.factorial(i + ell) for i in range(40))
    v = math.exp(z)
    for k in range(1, ell + 1):
        v = (v - 1.0 / math.factorial(k - 1)) / z
    return v


@pytest.mark.parametrize("n,scale,seed", [(5, 0.1, 0), (12, 3.0, 1), (20, 40.0, 2), (33, 300.0, 3)])
def test_expm_matches_scipy(n, scale, seed):
    X = wl.random_dense(n, seed, scale / math.sqrt(n))
    E = expm_pade13(X)
    R = scipy.linalg.expm(X)
    assert np.linalg.norm(E - R) / np.linalg.norm(R) < 1e-12


def test_expm_diagonal_closed_form():
    lam = np.array([-50.0, -3.0, -1e-3, 0.0, 0.5, 2.0])
    E = expm_pade13(np.diag(lam))
    assert np.allclose(np.diag(E), np.exp(lam), rtol=1e-14, atol=0)
    assert np.abs(E - np.diag(np.diag(E))).max() == 0.0


def test_expm_jordan_closed_form():
    # J = shift matrix (ones on the superdiagonal): e^{aI + J}_{i,i+k} = e^a / k!
    n, a = 7, -0.7
    X = a * np.eye(n) + np.diag(np.ones(n - 1), 1)
    E = expm_pade13(X)
    ref = np.zeros((n, n))
    for i in range(n):
        for k in range(n - i):
            ref[i, i + k] = math.exp(a) / math.factorial(k)
    assert np.abs(E - ref).max() < 1e-14


def test_pade_coefficients_closed_form():
    c = pade_coefficients(13)
    assert c[0] == 1.0 and abs(c[1] - 0.5) < 1e-16
    # p_13(x)/p_13(-x) agrees with e^x to O(x^27) near 0
    x = 0.05
    p = sum(c[j] * x**j for j in range(14))
    q = sum(c[j] * (-x)**j for j in range(14))
    assert abs(p / q - math.exp(x)) <= 4.5e-16 * math.exp(x)


@pytest.mark.parametrize("lmax", [1, 2, 3])
def test_phi_at_zero(lmax):
    # phi_l(0) = I / l!  (eq. (4b))
    n = 6
    ph = phi_matrices(np.zeros((n, n)), lmax)
    for ell, P in enumerate(ph):
        assert np.abs(P - np.eye(n) / math.factorial(ell)).max() < 1e-15


def test_phi_diagonal_scalar_closed_form():
    lam = np.array([-200.0, -7.5, -0.3, -1e-6, 0.0, 1e-6, 0.8, 3.0])
    ph = phi_matrices(np.diag(lam), 3)
    for ell in range(4):
        ref = np.array([scalar_phi(z, ell) for z in lam])
        assert np.allclose(np.diag(ph[ell]), ref, rtol=5e-14, atol=1e-300), ell


@pytest.mark.parametrize("n,eps,tau", [(9, 1.0, 1e-2), (17, 0.5, 1e-3), (31, 0.01, 1.0)])
def test_phi_dirichlet_laplacian_closed_form(n, eps, tau):
    """A = eps*D2 is S diag(lambda) S with S_jk = sqrt(2h) sin(jk pi h),
    lambda_k = -(4 eps/h^2) sin^2(k pi h / 2); phi_l(tau A) = S diag(phi_l(tau lambda)) S."""
    h = 1.0 / (n + 1)
    j = np.arange(1, n + 1)
    S = math.sqrt(2 * h) * np.sin(np.outer(j, j) * math.pi * h)
    lam = -(4 * eps / h**2) * np.sin(j * math.pi * h / 2) ** 2
    A = wl.fd_matrix(n, eps)
    assert np.abs(S @ np.diag(lam) @ S - A).max() < 1e-9 * np.abs(A).max()
    ph = phi_matrices(tau * A, 2)
    for ell in range(3):
        ref = S @ np.diag([scalar_phi(tau * l, ell) for l in lam]) @ S
        assert np.abs(ph[ell] - ref).max() < 1e-13, ell


def test_phi_squaring_recurrence_eq16():
    """phi_l(2X) = 2^-l [e^X phi_l(X) + sum_{k=1}^l phi_k(X)/(l-k)!]  (eq. (16))."""
    X = wl.random_dense(10, 7, 0.6)
    ph = phi_matrices(X, 3)
    ph2 = phi_matrices(2 * X, 3)
    for ell in range(1, 4):
        rhs = ph[0] @ ph[ell]
        for k in range(1, ell + 1):
            rhs = rhs + ph[k] / math.factorial(ell - k)
        rhs = rhs / 2**ell
        assert np.abs(ph2[ell] - rhs).max() < 1e-13 * max(1.0, np.abs(rhs).max())


def test_phi_integral_definition_eq4a():
    """phi_l(X) = 1/(l-1)! int_0^1 e^{(1-theta)X} theta^{l-1} dtheta, by Gauss-Legendre
    quadrature of scipy's expm (an independent route)."""
    X = wl.random_dense(8, 11, 0.5)
    nodes, weights = np.polynomial.legendre.leggauss(30)
    th = 0.5 * (nodes + 1.0)
    w = 0.5 * weights
    ph = phi_matrices(X, 2)
    for ell in (1, 2):
        ref = sum(wi * scipy.linalg.expm((1 - t) * X) * t ** (ell - 1)
                  for t, wi in zip(th, w)) / math.factorial(ell - 1)
        assert np.abs(ph[ell] - ref).max() < 1e-13


def test_phi_adr_matrix_vs_scipy_augmented():
    # phi_1, phi_2 of a nonsymmetric ADR matrix with tau*||A|| >> 1, against
    # scipy's expm of the same augmented matrix built by hand here.
    n = 40
    A = wl.fd_matrix(n, 0.5, 1.0)
    X = 1e-3 * A
    ph = phi_matrices(X, 2)
    Z = np.zeros((3 * n, 3 * n))
    Z[:n, :n] = X
    Z[:n, n:2 * n] = np.eye(n)
    Z[n:2 * n, 2 * n:] = np.eye(n)
    E = scipy.linalg.expm(Z)
    for ell in range(3):
        ref = E[:n, ell * n:(ell + 1) * n]
        assert np.abs(ph[ell] - ref).max() < 1e-13 * max(1, np.abs(ref).max())
