"""Seeded synthetic problems in Kronecker form (Section 1, eq. (1)-(3); Section 4).

This module holds the *problem data* that both the CUDA path and the FP64 oracle
consume: the small matrices A_mu, the initial state, the nonlinearity's
coefficients, the step size and the step count.  It contains none of the method's
arithmetic (no phi-function, no mu-mode product, no integrator); it only builds
inputs from seeds, so the two implementations share data, never code.

Layout convention (Section 1, the vec operator stacks columns; A_1 acts on the
fastest index i_1): an order-d state tensor of sizes n_1 x ... x n_d is stored as a
numpy array of shape (n_d, ..., n_1), C-contiguous, so that the flat memory order
is i_1 fastest.  All matrices are n x n float64, C-contiguous with
M[i, j] = entry (i, j); the CUDA library receives them column-major (that is, the
transpose buffer) through ``to_colmajor``.

Spatial discretisation (Section 4.2, second-order centred differences on the
inner points of [0, 1] with homogeneous Dirichlet boundaries, h = 1/(n+1)):
    D2 = h^-2 tridiag(1, -2, 1),    D1 = (2h)^-1 tridiag(-1, 0, 1),
    A  = eps * D2 + beta * D1.

Input recipe of each workload is stated in its docstring.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# Nonlinearity kinds understood by both sides.
G_NONE = 0      # g = 0
G_CUBIC = 1     # g(u) = c0 + c1 u + c2 u^2 + c3 u^3, pointwise
G_RICCATI = 2   # G(U) = C + U B U (Section 1, eq. (2))
G_ADR_MANUFACTURED = 3  # g(t,u) = 1/(1+u^2) + Psi(t, x), Section 4.2 (eq. (25))

EXPEULER = 0    # exponential Euler, eq. (11); tensor form eq. (19)
ETD2RK = 1      # ETD2RK, eq. (12); tensor form eq. (20)
LAWSON_EULER = 2  # Lawson-Euler, eq. (9); tensor form eq. (17)
LAWSON2B = 3    # Lawson2b, eq. (10); tensor form eq. (18)
EXPROSEULER = 4  # exponential Rosenbrock-Euler, eq. (13); tensor form eq. (21) (Riccati)
EXPEULER_ALT = 5  # exponential Euler, alternative form (Section 3.2)

SCHEME_NAMES = {EXPEULER: "expeuler", ETD2RK: "etd2rk",
                LAWSON_EULER: "lawson_euler", LAWSON2B: "lawson2b", EXPROSEULER: "exprosenbrock",
                EXPEULER_ALT: "expeuler_alt"}


@dataclasses.dataclass
class Problem:
    """u' = K u + g(t, u) with K = A_d (+) ... (+) A_1 (eq. (1a)-(1b))."""
    name: str
    A: List[np.ndarray]            # A[mu-1] is n_mu x n_mu, float64
    u0: np.ndarray                 # shape (n_d, ..., n_1), float64
    g_kind: int = G_NONE
    cubic: Sequence[float] = (0.0, 0.0, 0.0, 0.0)
    B: Optional[np.ndarray] = None  # Riccati B (n_2 x n_1)
    C: Optional[np.ndarray] = None  # Riccati C (n_1 x n_2), stored like u0: shape (n_2, n_1)
    # Manufactured forcing Psi(t) = e^t psi_a - 1/(1 + e^{2t} psi_b^2) (same shape as u0).
    psi_a: Optional[np.ndarray] = None
    psi_b: Optional[np.ndarray] = None
    tau: float = 1e-3
    steps: int = 1
    scheme: int = EXPEULER

    @property
    def d(self) -> int:
        return len(self.A)

    @property
    def n(self) -> List[int]:
        return [a.shape[0] for a in self.A]

    @property
    def N(self) -> int:
        return int(np.prod(self.n))


def grid(n: int) -> np.ndarray:
    """Inner grid points x_i = i h, i = 1..n, h = 1/(n+1)."""
    h = 1.0 / (n + 1)
    return h * np.arange(1, n + 1, dtype=np.float64)


def fd_matrix(n: int, eps: float, beta: float = 0.0) -> np.ndarray:
    """A = eps*D2 + beta*D1 on n inner points, Dirichlet (Section 4.2)."""
    h = 1.0 / (n + 1)
    A = np.zeros((n, n), dtype=np.float64)
    i = np.arange(n)
    A[i, i] = -2.0 * eps / h**2
    A[i[1:], i[1:] - 1] = eps / h**2 - beta / (2.0 * h)
    A[i[:-1], i[:-1] + 1] = eps / h**2 + beta / (2.0 * h)
    return A


def to_colmajor(M: np.ndarray) -> np.ndarray:
    """Return a C-contiguous buffer holding M in column-major order (M^T)."""
    return np.ascontiguousarray(M.T)


def allen_cahn_2d(n: int = 64, eps: float = 0.01, seed: int = 1, tau: float = 1e-3,
                  steps: int = 50, scheme: int = EXPEULER) -> Problem:
    """2D Allen-Cahn u' = eps*Lap(u) + u - u^3 on [0,1]^2, Dirichlet.

    K = eps * Lap_h (both directions), g(u) = u - u^3 pointwise; u0 i.i.d.
    uniform in [-0.9, 0.9] drawn from ``seed`` (numpy PCG64).
    """
    rng = np.random.default_rng(seed)
    A = fd_matrix(n, eps)
    u0 = rng.uniform(-0.9, 0.9, size=(n, n))
    return Problem(name=f"allen_cahn_2d_n{n}", A=[A, A.copy()], u0=u0,
                   g_kind=G_CUBIC, cubic=(0.0, 1.0, 0.0, -1.0), tau=tau,
                   steps=steps, scheme=scheme)


def adr_3d(n: int = 128, eps: float = 0.5, beta: float = 1.0, seed: int = 2,
           tau: float = 1e-3, steps: int = 100, scheme: int = ETD2RK,
           noise: float = 1e-3, sizes: Optional[Sequence[int]] = None) -> Problem:
    """3D advection-diffusion-reaction u' = eps*Lap(u) + beta.grad(u) + u(u-1/2)(1-u).

    A_mu = eps*D2 + beta*D1 per direction; g(u) = u(u-1/2)(1-u)
    = -0.5 u + 1.5 u^2 - u^3; u0 = 64 prod x_mu (1 - x_mu) (the bump of Section
    4.2) plus i.i.d. uniform noise in [-noise, noise] drawn from ``seed``.
    ``sizes`` overrides (n_1, n_2, n_3) for non-cubic grids.
    """
    ns = list(sizes) if sizes is not None else [n, n, n]
    A = [fd_matrix(m, eps, beta) for m in ns]
    x1, x2, x3 = (grid(m) for m in ns)
    bump = 64.0 * ((x3 * (1 - x3))[:, None, None] * (x2 * (1 - x2))[None, :, None]
                   * (x1 * (1 - x1))[None, None, :])
    rng = np.random.default_rng(seed)
    u0 = bump + rng.uniform(-noise, noise, size=bump.shape)
    return Problem(name="adr_3d_n" + "x".join(map(str, ns)), A=A, u0=u0,
                   g_kind=G_CUBIC, cubic=(0.0, -0.5, 1.5, -1.0), tau=tau,
                   steps=steps, scheme=scheme)


def riccati_2d(n: int = 2048, seed: int = 5, tau: float = 1e-4, steps: int = 50,
               scheme: int = EXPEULER, skew: float = 0.1, sigma: float = 1e-2) -> Problem:
    """Matrix Riccati U' = A1 U + U A2^T + C + U B U, U0 = 0 (eq. (2); Kronecker form eq. (3)).

    A_mu = h^-2 tridiag(1,-2,1) + skew * S_mu, h = 1/(n+1), S_mu = (G - G^T)/sqrt(2)
    with G i.i.d. N(0,1); B, C i.i.d. N(0, sigma^2).  Independent streams for
    A1, A2, B, C come from ``seed`` via numpy SeedSequence.spawn.
    """
    ss = np.random.SeedSequence(seed).spawn(4)
    rngs = [np.random.default_rng(s) for s in ss]
    D2 = fd_matrix(n, 1.0)
    A = []
    for r in rngs[:2]:
        G = r.standard_normal((n, n))
        A.append(D2 + skew * (G - G.T) / math.sqrt(2.0))
    B = sigma * rngs[2].standard_normal((n, n))      # B[i, j], n_2 x n_1
    Cm = sigma * rngs[3].standard_normal((n, n))     # C[i1, i2]
    # States are stored as (n_2, n_1) arrays (i_1 fastest): U_store = U^T.
    return Problem(name=f"riccati_2d_n{n}", A=A, u0=np.zeros((n, n)),
                   g_kind=G_RICCATI, B=B, C=np.ascontiguousarray(Cm.T), tau=tau,
                   steps=steps, scheme=scheme)


def lq_operators(nhat: int, alpha: float = 100.0):
    """The pieces of the paper's linear-quadratic control problem (Section 4.1).

    On the inner nhat x nhat grid x_i = i h, h = 1/(nhat + 1), with homogeneous
    Dirichlet conditions and second-order centred differences:
      D1 = discretisation of d_xx - 10 x d_x,   D2 = of d_yy - 100 y d_y (nhat x nhat),
      A  = I (x) D1 + D2 (x) I (n x n, n = nhat^2, unknown k = i + (j - 1) nhat),
    b_k = 1 where 0.1 < x_i <= 0.3, c_k = 1 where 0.7 < x_i <= 0.9, B = -b b^T,
    C = alpha c^T c.  Returns (D1, D2, A, B, C)."""
    h = 1.0 / (nhat + 1)
    x = grid(nhat)

    def d1(coef):
        D = np.zeros((nhat, nhat))
        for i in range(nhat):
            D[i, i] = -2.0 / h ** 2
            if i > 0:
                D[i, i - 1] = 1.0 / h ** 2 + coef * x[i] / (2 * h)
            if i < nhat - 1:
                D[i, i + 1] = 1.0 / h ** 2 - coef * x[i] / (2 * h)
        return D

    D1, D2 = d1(10.0), d1(100.0)
    I = np.eye(nhat)
    A = np.kron(I, D1) + np.kron(D2, I)
    xi = np.tile(x, nhat)                                # x_i of unknown k
    b = ((xi > 0.1) & (xi <= 0.3)).astype(np.float64)
    c = ((xi > 0.7) & (xi <= 0.9)).astype(np.float64)
    return D1, D2, A, -np.outer(b, b), alpha * np.outer(c, c)


def lq_riccati(nhat: int = 30, steps: int = 170, scheme: int = ETD2RK, T: float = 0.025,
               alpha: float = 100.0) -> Problem:
    """The paper's linear-quadratic control problem (Section 4.1), no random input.

    A (n x n, n = nhat^2) discretises d_xx + d_yy - 10 x d_x - 100 y d_y (see
    lq_operators); U0 = 0.  The Riccati equation U' = A^T U + U A + C + U B U is the
    two-direction form with A_1 = A_2 = A^T; tau = T / steps.
    """
    _, _, A, B, Cm = lq_operators(nhat, alpha)
    n = nhat * nhat
    return Problem(name=f"lq_riccati_nhat{nhat}", A=[A.T.copy(), A.T.copy()], u0=np.zeros((n, n)),
                   g_kind=G_RICCATI, B=B, C=np.ascontiguousarray(Cm.T), tau=T / steps,
                   steps=steps, scheme=scheme)


def lq_riccati_order4(nhat: int = 30, steps: int = 170, scheme: int = ETD2RK, T: float = 0.025,
                      alpha: float = 100.0) -> Problem:
    """The same LQ problem in the order-4 tensor form of the remark closing Section 4.1.

    A^T = I (x) D1^T + D2^T (x) I is itself a Kronecker sum, so A^T U + U A is the
    four-direction Kronecker sum K = A_4 (+) A_3 (+) A_2 (+) A_1 with A_1 = A_3 = D1^T
    and A_2 = A_4 = D2^T (nhat x nhat each) acting on U as an nhat^4 tensor: i_1, i_2
    the x and y indices of the matrix row k = i_1 + nhat i_2, i_3, i_4 those of the
    column.  The state's memory layout is the two-direction form's (the column-major
    n x n matrix); G(U) = C + U B U is formed on that matrix view.
    """
    D1, D2, _, B, Cm = lq_operators(nhat, alpha)
    sh = (nhat,) * 4
    return Problem(name=f"lq_riccati_order4_nhat{nhat}",
                   A=[D1.T.copy(), D2.T.copy(), D1.T.copy(), D2.T.copy()], u0=np.zeros(sh),
                   g_kind=G_RICCATI, B=B, C=np.ascontiguousarray(Cm.T).reshape(sh), tau=T / steps,
                   steps=steps, scheme=scheme)


def paper_adr_3d(sizes: Sequence[int] = (40, 41, 42), steps: int = 40,
                 scheme: int = ETD2RK, eps: float = 0.75, alpha: float = 0.1,
                 T: float = 1.0) -> Problem:
    """The paper's own ADR test (Section 4.2, eq. (25)), no random input.

    u_t = eps Lap u + alpha (d_1 + d_2 + d_3) u + 1/(1+u^2) + Psi on [0,1]^3,
    Dirichlet, u0 = 64 prod f(x_mu), f(x) = x(1-x); Psi makes u = e^t u0 exact.
    Because u0 is a product of quadratics, the centred differences are exact on
    it, so Psi is written from the PDE with exact derivatives of u0:
        Psi(t) = e^t (u0 - eps Lap u0 - alpha sum_mu d_mu u0) - 1/(1 + e^{2t} u0^2),
    stored as psi_a = u0 - eps Lap u0 - alpha sum d_mu u0 and psi_b = u0.
    The exact solution of the semi-discrete system at T is e^T u0.
    """
    ns = list(sizes)
    A = [fd_matrix(m, eps, alpha) for m in ns]
    x1, x2, x3 = (grid(m) for m in ns)
    f = [x * (1 - x) for x in (x1, x2, x3)]
    fp = [1 - 2 * x for x in (x1, x2, x3)]
    fpp = [-2.0 * np.ones_like(x) for x in (x1, x2, x3)]

    def prod(a1, a2, a3):   # a_mu along i_mu, tensor shape (n3, n2, n1)
        return a3[:, None, None] * a2[None, :, None] * a1[None, None, :]

    u0 = 64.0 * prod(f[0], f[1], f[2])
    lap = 64.0 * (prod(fpp[0], f[1], f[2]) + prod(f[0], fpp[1], f[2]) + prod(f[0], f[1], fpp[2]))
    div = 64.0 * (prod(fp[0], f[1], f[2]) + prod(f[0], fp[1], f[2]) + prod(f[0], f[1], fp[2]))
    return Problem(name="paper_adr_3d_" + "x".join(map(str, ns)), A=A, u0=u0,
                   g_kind=G_ADR_MANUFACTURED, psi_a=u0 - eps * lap - alpha * div,
                   psi_b=u0.copy(), tau=T / steps, steps=steps, scheme=scheme)


BATCH_SIZES = tuple(range(48, 513, 16))   # {48, 64, ..., 512}: 30 values


def batched_allen_cahn(count: int = 1024, seed: int = 4, tau: float = 1e-3,
                       steps: int = 20, sizes: Sequence[int] = BATCH_SIZES,
                       eps_range=(1e-3, 1e-1)) -> List[Problem]:
    """Independent 2D Allen-Cahn instances of uneven size.

    Instance k: n_k uniform over ``sizes``, eps_k log-uniform in ``eps_range``,
    u0 i.i.d. uniform in [-0.9, 0.9]; exponential Euler.  One PCG64 stream from
    ``seed`` draws (n_k, eps_k) for all k first, then the initial states in order.
    """
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=count)
    le = rng.uniform(math.log(eps_range[0]), math.log(eps_range[1]), size=count)
    probs = []
    for k in range(count):
        n = int(ns[k])
        A = fd_matrix(n, float(math.exp(le[k])))
        u0 = rng.uniform(-0.9, 0.9, size=(n, n))
        probs.append(Problem(name=f"ac2d_batch{k}_n{n}", A=[A, A.copy()], u0=u0,
                             g_kind=G_CUBIC, cubic=(0.0, 1.0, 0.0, -1.0), tau=tau,
                             steps=steps, scheme=EXPEULER))
    return probs


def random_dense(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """i.i.d. N(0, scale^2) n x n matrix (test inputs)."""
    return scale * np.random.default_rng(seed).standard_normal((n, n))


def random_tensor(shape: Sequence[int], seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """i.i.d. uniform tensor (test inputs); ``shape`` is (n_d, ..., n_1)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=tuple(shape))


# The workloads of the measured configurations, named by what they are.
def workload(name: str, **over) -> Problem:
    table = {
        "ac2d_n64_expeuler": lambda: allen_cahn_2d(64, 0.01, 1, 1e-3, 50, EXPEULER),
        "adr3d_n128_etd2rk": lambda: adr_3d(128, 0.5, 1.0, 2, 1e-3, 100, ETD2RK),
        "adr3d_n320_etd2rk": lambda: adr_3d(320, 0.5, 1.0, 3, 1e-3, 100, ETD2RK),
        # the same problem at n = 256 (N = 16.8M, operands still larger than L2): the
        # size on which kernel profiles are captured
        "adr3d_n256_etd2rk": lambda: adr_3d(256, 0.5, 1.0, 3, 1e-3, 100, ETD2RK),
        "riccati_n2048_expeuler": lambda: riccati_2d(2048, 5, 1e-4, 50, EXPEULER),
        "riccati_n2048_etd2rk": lambda: riccati_2d(2048, 5, 1e-4, 50, ETD2RK),
        # the paper's LQ-control problem (Section 4.1), nhat = 30, T = 0.025, 170 steps
        "lq_riccati_nhat30_etd2rk": lambda: lq_riccati(30, 170, ETD2RK),
        "lq_riccati_nhat30_exprosenbrock": lambda: lq_riccati(30, 170, EXPROSEULER),
        # the same problem as an order-4 tensor with the 30 x 30 matrices D1^T, D2^T
        # (the remark closing Section 4.1)
        "lq_riccati_order4_nhat30_etd2rk": lambda: lq_riccati_order4(30, 170, ETD2RK),
    }
    if name in BATCHED:
        raise ValueError(f"{name} is a batch: use batched_workload()")
    p = table[name]()
    for k, v in over.items():
        setattr(p, k, v)
    return p


# Batches of independent problems, named by what they are.
BATCHED = {
    "batch_ac2d_1024_expeuler": lambda: batched_allen_cahn(1024, 4, 1e-3, 20),
    # the first 256 instances of the same draw: the size on which kernel profiles are
    # captured (about 2 GB on the device with the comparison loop's plans)
    "batch_ac2d_256_expeuler": lambda: batched_allen_cahn(1024, 4, 1e-3, 20)[:256],
}


def batched_workload(name: str) -> List[Problem]:
    return BATCHED[name]()
