"""mu-mode product, Tucker operator and the split phi action (oracle; test infrastructure).

Tensors are numpy arrays of shape (n_d, ..., n_1), C-contiguous, so the flat order
is i_1 fastest (the vec of Section 1).  Direction mu therefore lives on numpy
axis d - mu.

* mu-mode product (Section 1, eq. (7) factorised one direction at a time):
      (V x_mu M)[..., i_mu, ...] = sum_j M[i_mu, j] V[..., j, ...].
* Tucker operator (eq. (6)): V x_1 M_1 x_2 M_2 ... x_d M_d, in that order.
* PHISPLIT (Section 3, Theorem 1 / eq. (14) and the definition of P_l^(2) after it):
      P_l^(2) = ((l!)^(d-1) V) x_1 phi_l(tau A_1) ... x_d phi_l(tau A_d).
"""
from __future__ import annotations

import math

import numpy as np


def mode_product(V: np.ndarray, M: np.ndarray, mu: int) -> np.ndarray:
    """V x_mu M, mu = 1..d (contraction of M's column index with index i_mu)."""
    d = V.ndim
    axis = d - mu
    Y = np.tensordot(M, V, axes=([1], [axis]))     # new index i_mu first
    return np.ascontiguousarray(np.moveaxis(Y, 0, axis))


def tucker(V: np.ndarray, Ms) -> np.ndarray:
    """V x_1 Ms[0] x_2 Ms[1] ... x_d Ms[d-1]."""
    Y = np.asarray(V, dtype=np.float64)
    for mu, M in enumerate(Ms, start=1):
        Y = mode_product(Y, M, mu)
    return Y


def phisplit_apply(V: np.ndarray, phis, ell: int) -> np.ndarray:
    """P_l^(2) = ((l!)^(d-1) V) x_1 phis[0] ... x_d phis[d-1]  (Section 3).

    ``phis[mu-1]`` must be phi_l(tau A_mu).  For l = 0 this is the exact
    e^{tau K} v of eq. (5)-(6) (the factor is 1).
    """
    d = V.ndim
    scale = float(math.factorial(ell)) ** (d - 1)
    return tucker(scale * np.asarray(V, dtype=np.float64), phis)


def phisplit_apply_at(V: np.ndarray, phis, ell: int, index_sets) -> np.ndarray:
    """The entries of P_l^(2) on the grid index_sets[0] x ... x index_sets[d-1]
    (index_sets[mu-1] lists values of i_mu), for checks on tensors too large to
    transform in full.  Restricting the output index i_mu of a mu-mode product to a
    set I is the mu-mode product with the rows I of the matrix, so this is the
    same Tucker chain (Section 3) with phis[mu-1][I_mu, :].  Result shape:
    (|I_d|, ..., |I_1|)."""
    rows = [np.asarray(phi)[np.asarray(I, dtype=np.int64), :] for phi, I in zip(phis, index_sets)]
    return phisplit_apply(V, rows, ell)
