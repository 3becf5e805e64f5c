"""K u, g(u) and the PHISPLIT time steppers, FP64 (oracle; test infrastructure).

Tensor formulations of Section 3.2 with tensors in the (n_d, ..., n_1) layout:

* K u without assembling K:  sum_mu U x_mu A_mu                 (Section 3.2)
* exponential Euler (eq. (19)):
      U+ = U + tau * (K U + G(U)) x_1 phi_1(tau A_1) ... x_d phi_1(tau A_d)
* ETD2RK (eq. (20), read with tau multiplying both K U and G, as the vector form
  eq. (12) requires, and with the (2!)^(d-1) factor of P_2^(2) from Theorem 1):
      U2 = U  + tau * P_1^(2)(K U + G(U))
      U+ = U2 + tau * P_2^(2)(G(U2) - G(U))
  where P_l^(2)(V) = ((l!)^(d-1) V) x_1 phi_l(tau A_1) ... x_d phi_l(tau A_d).
* Lawson-Euler (eq. (17)):  U+ = (U + tau G(U)) x_mu e^{tau A_mu}
* Lawson2b (eq. (18)):
      U2 = (U + tau G(U)) x_mu e^{tau A_mu}
      U+ = (U + tau/2 G(U)) x_mu e^{tau A_mu} + tau/2 G(U2)
* exponential Euler, alternative form (Section 3.2, after eq. (19)), exact for
  linear autonomous problems:
      U+ = U x_mu e^{tau A_mu} + tau * G(U) x_1 phi_1(tau A_1) ... x_d phi_1(tau A_d)
* exponential Rosenbrock-Euler (eq. (13), tensor form eq. (21), read like eq. (20)
  with tau on both K U and G), for the Riccati term only, whose Jacobian at U_n is
  again a Kronecker sum (Section 4.1): J_1 = A_1 + U_n B, J_2 = A_2 + (B U_n)^T and
      U+ = U + tau * (K U + G(U)) x_1 phi_1(tau J_1) x_2 phi_1(tau J_2)

g may depend on t only through the manufactured forcing of the paper's ADR test
(Section 4.2): g(t, u) = 1/(1 + u^2) + e^t a - 1/(1 + e^{2t} b^2), with the
arrays a, b supplied by the caller.  Stage times follow eq. (9)-(12): G(t_n, U_n)
and, for the second stages, G(t_{n+1}, U_n2).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

from .phi import phi_matrices
from .tucker import mode_product, phisplit_apply, phisplit_apply_at

G_NONE, G_CUBIC, G_RICCATI, G_ADR_MANUFACTURED = 0, 1, 2, 3
EXPEULER, ETD2RK, LAWSON_EULER, LAWSON2B, EXPROSEULER, EXPEULER_ALT = 0, 1, 2, 3, 4, 5


@dataclasses.dataclass
class OracleProblem:
    """Everything one integration needs; built by the caller from plain arrays."""
    A: List[np.ndarray]
    tau: float
    g_kind: int = G_NONE
    cubic: Sequence[float] = (0.0, 0.0, 0.0, 0.0)
    B: Optional[np.ndarray] = None
    C: Optional[np.ndarray] = None
    psi_a: Optional[np.ndarray] = None
    psi_b: Optional[np.ndarray] = None
    phis: Optional[List[List[np.ndarray]]] = None   # phis[mu-1][l] = phi_l(tau A_mu)

    def ensure_phis(self, lmax: int = 2) -> None:
        if self.phis is None or len(self.phis[0]) <= lmax:
            self.phis = [phi_matrices(self.tau * A, lmax) for A in self.A]

    def phi_list(self, ell: int) -> List[np.ndarray]:
        return [p[ell] for p in self.phis]

    @classmethod
    def from_problem(cls, p, lmax: int = 2) -> "OracleProblem":
        op = cls(A=[np.asarray(a, dtype=np.float64) for a in p.A], tau=float(p.tau),
                 g_kind=p.g_kind, cubic=tuple(p.cubic), B=p.B, C=p.C,
                 psi_a=getattr(p, "psi_a", None), psi_b=getattr(p, "psi_b", None))
        op.ensure_phis(lmax)
        return op


def kron_apply(U: np.ndarray, A: Sequence[np.ndarray]) -> np.ndarray:
    """K u in tensor form: sum_mu U x_mu A_mu (Section 3.2)."""
    out = np.zeros_like(U, dtype=np.float64)
    for mu, Amu in enumerate(A, start=1):
        out += mode_product(U, Amu, mu)
    return out


def g_eval(op: OracleProblem, U: np.ndarray, t: float = 0.0) -> np.ndarray:
    """G(t, U): zero, a pointwise cubic, the Riccati term C + U B U (eq. (2)),
    or the manufactured ADR nonlinearity of Section 4.2."""
    if op.g_kind == G_NONE:
        return np.zeros_like(U)
    if op.g_kind == G_CUBIC:
        c0, c1, c2, c3 = op.cubic
        return c0 + c1 * U + c2 * U * U + c3 * U * U * U
    if op.g_kind == G_RICCATI:
        # The state is the matrix U whose column-stacked vec is the tensor's (Section
        # 1): rows = the first d/2 directions, columns = the rest (d = 2: n_1 x n_2;
        # d = 4, the order-4 form of the Section 4.1 remark: n_1 n_2 x n_3 n_4).
        # Stored arrays are C-ordered (n_d, ..., n_1), i.e. transposes of the matrices.
        m1 = int(np.prod(U.shape[U.ndim // 2:]))
        m2 = U.size // m1
        Um = U.reshape(m2, m1).T
        Cm = op.C.reshape(m2, m1).T
        return np.ascontiguousarray((Cm + Um @ op.B @ Um).T).reshape(U.shape)
    if op.g_kind == G_ADR_MANUFACTURED:
        et = np.exp(t)
        return (1.0 / (1.0 + U * U) + et * op.psi_a
                - 1.0 / (1.0 + et * et * op.psi_b * op.psi_b))
    raise ValueError(f"unknown g kind {op.g_kind}")


def riccati_jacobian(op: OracleProblem, U: np.ndarray) -> List[np.ndarray]:
    """[J_1, J_2] with K + dG(U) = J_2 (+) J_1 for G(U) = C + U B U (Section 4.1):
    the derivative V B U + U B V of U B U adds U B to A_1 and (B U)^T to A_2."""
    Um = U.T                      # stored arrays are (n_2, n_1): the transposes
    return [op.A[0] + Um @ op.B, op.A[1] + (op.B @ Um).T]


def step(op: OracleProblem, U: np.ndarray, scheme: int, t: float = 0.0) -> np.ndarray:
    """One step of size op.tau from (t, U) (Section 3.2 tensor formulations)."""
    tau = op.tau
    if scheme == EXPEULER:
        W = kron_apply(U, op.A) + g_eval(op, U, t)
        return U + tau * phisplit_apply(W, op.phi_list(1), 1)
    if scheme == ETD2RK:
        Gn = g_eval(op, U, t)
        W1 = kron_apply(U, op.A) + Gn
        U2 = U + tau * phisplit_apply(W1, op.phi_list(1), 1)
        W2 = g_eval(op, U2, t + tau) - Gn
        return U2 + tau * phisplit_apply(W2, op.phi_list(2), 2)
    if scheme == LAWSON_EULER:
        return phisplit_apply(U + tau * g_eval(op, U, t), op.phi_list(0), 0)
    if scheme == LAWSON2B:
        Gn = g_eval(op, U, t)
        U2 = phisplit_apply(U + tau * Gn, op.phi_list(0), 0)
        return (phisplit_apply(U + 0.5 * tau * Gn, op.phi_list(0), 0)
                + 0.5 * tau * g_eval(op, U2, t + tau))
    if scheme == EXPEULER_ALT:
        return (phisplit_apply(U, op.phi_list(0), 0)
                + tau * phisplit_apply(g_eval(op, U, t), op.phi_list(1), 1))
    if scheme == EXPROSEULER:
        if op.g_kind != G_RICCATI:
            raise ValueError("exponential Rosenbrock-Euler needs the Riccati term")
        W = kron_apply(U, op.A) + g_eval(op, U, t)
        phis = [phi_matrices(tau * J, 1)[1] for J in riccati_jacobian(op, U)]
        return U + tau * phisplit_apply(W, phis, 1)
    raise ValueError(f"unknown scheme {scheme}")


def step_at(op: OracleProblem, U: np.ndarray, scheme: int, t: float, index_sets) -> np.ndarray:
    """The entries of step(op, U, scheme, t) on the grid index_sets[0] x ... x
    index_sets[d-1] (index_sets[mu-1] lists values of i_mu), for checks on states
    too large to step in full.  Every tensor the step needs in full -- K U + G(U),
    and for ETD2RK the first stage U2 and G(U2) - G(U) -- is formed in full; only
    the last Tucker operator of the step is restricted to the sampled rows of its
    phi matrices (phisplit_apply_at).  Exponential Euler (eq. (19)), ETD2RK
    (eq. (20)) and Lawson-Euler (eq. (17)).  Result shape (|I_d|, ..., |I_1|)."""
    tau = op.tau
    ix = np.ix_(*[np.asarray(I, dtype=np.int64) for I in reversed(list(index_sets))])
    if scheme == EXPEULER:
        W = kron_apply(U, op.A) + g_eval(op, U, t)
        return U[ix] + tau * phisplit_apply_at(W, op.phi_list(1), 1, index_sets)
    if scheme == ETD2RK:
        Gn = g_eval(op, U, t)
        W1 = kron_apply(U, op.A) + Gn
        U2 = U + tau * phisplit_apply(W1, op.phi_list(1), 1)
        W2 = g_eval(op, U2, t + tau) - Gn
        return U2[ix] + tau * phisplit_apply_at(W2, op.phi_list(2), 2, index_sets)
    if scheme == LAWSON_EULER:
        return phisplit_apply_at(U + tau * g_eval(op, U, t), op.phi_list(0), 0, index_sets)
    raise ValueError(f"step_at: scheme {scheme} not supported")


def integrate(op: OracleProblem, U0: np.ndarray, scheme: int, nsteps: int,
              t0: float = 0.0) -> np.ndarray:
    """nsteps constant-size steps from (t0, U0)."""
    op.ensure_phis(2)
    U = np.array(U0, dtype=np.float64, copy=True)
    for k in range(nsteps):
        U = step(op, U, scheme, t0 + k * op.tau)
    return U


def rel_err_inf(x: np.ndarray, ref: np.ndarray) -> float:
    """||x - ref||_inf / ||ref||_inf (the ADR convention of Section 4.2)."""
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(x - ref)) / (den if den > 0 else 1.0))


def rel_err_fro(x: np.ndarray, ref: np.ndarray) -> float:
    """||x - ref||_F / ||ref||_F (the Riccati convention of Section 4.1)."""
    den = np.linalg.norm(ref.ravel())
    return float(np.linalg.norm((x - ref).ravel()) / (den if den > 0 else 1.0))
