"""Small-matrix exponential and phi-functions, FP64 (oracle; test infrastructure).

phi-functions (Section 1, eq. (4a)-(4b)):
    phi_0(X) = e^X,   phi_l(X) = sum_{i>=0} X^i / (i+l)!.

e^X: diagonal Pade [13/13] approximant with scaling and squaring, the method the
paper uses for phi_0 (Section 3.1, ``expm`` of Al-Mohy and Higham; the [13/13]
degree and the scaling threshold theta_13 are those of Higham, SIAM J. Matrix
Anal. Appl. 26 (2005) 1179-1193, Table 2.3).  Pade coefficients come from the
closed form c_j = (2m-j)! m! / ((2m)! j! (m-j)!).

phi_1..phi_lmax: exponential of the block upper-triangular augmented matrix
    X_aug = [[X, I, 0, ...], [0, 0, I, ...], ..., [0, ..., 0]]  (lmax+1 blocks),
whose exponential has e^X, phi_1(X), ..., phi_lmax(X) as its first block row.
This identity follows from the series (eq. (4b)): the first block row of X_aug^k
is (X^k, X^(k-1), ..., X^(k-lmax)), so block (1, l+1) of e^{X_aug} is
sum_k X^(k-l)/k! = phi_l(X).  It is a different route from the GPU plan
(scaled Taylor plus the squaring recurrence of eq. (16)), so the two check each
other.
"""
from __future__ import annotations

import math

import numpy as np

PADE13_THETA = 5.371920351148152   # Higham (2005), Table 2.3, m = 13
PADE_M = 13


def pade_coefficients(m: int = PADE_M) -> np.ndarray:
    """c_j, j = 0..m, of the [m/m] Pade numerator p_m(x) = sum c_j x^j."""
    f = math.factorial
    return np.array([f(2 * m - j) * f(m) / (f(2 * m) * f(j) * f(m - j))
                     for j in range(m + 1)], dtype=np.float64)


def expm_pade13(X: np.ndarray) -> np.ndarray:
    """e^X by Pade [13/13] + scaling and squaring, plain FP64.

    1. s = smallest integer >= 0 with ||X / 2^s||_1 <= theta_13.
    2. Y = X / 2^s; powers Y^0..Y^13 formed one product at a time.
    3. p = sum c_j Y^j, q = sum c_j (-Y)^j, R = q^{-1} p (a linear solve).
    4. square R s times.
    """
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    norm1 = np.abs(X).sum(axis=0).max() if n else 0.0
    s = 0
    if norm1 > PADE13_THETA:
        s = int(math.ceil(math.log2(norm1 / PADE13_THETA)))
    Y = X / (2.0 ** s)
    c = pade_coefficients(PADE_M)
    P = np.zeros_like(Y)
    Q = np.zeros_like(Y)
    Yj = np.eye(n)
    for j in range(PADE_M + 1):
        P += c[j] * Yj
        Q += ((-1.0) ** j) * c[j] * Yj
        Yj = Yj @ Y
    R = np.linalg.solve(Q, P)
    for _ in range(s):
        R = R @ R
    return R


def phi_matrices(X: np.ndarray, lmax: int) -> list:
    """[phi_0(X), phi_1(X), ..., phi_lmax(X)] via e^{X_aug} (see module doc)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    m = (lmax + 1) * n
    Xa = np.zeros((m, m), dtype=np.float64)
    Xa[:n, :n] = X
    for b in range(lmax):
        Xa[b * n:(b + 1) * n, (b + 1) * n:(b + 2) * n] = np.eye(n)
    E = expm_pade13(Xa)
    return [E[:n, b * n:(b + 1) * n].copy() for b in range(lmax + 1)]
