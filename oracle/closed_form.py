"""Closed forms of S_k(A) and of the radix-framework result, and probe Horner.

For a planted symmetric A = Q diag(lam) Q^T (Q = H_1 ... H_r, Householder
reflectors H_i = I - 2 v_i v_i^T / v_i^T v_i), any polynomial p(A) equals
Q diag(p(lam)) Q^T, so the matrix result is fixed by a scalar function:

  * S_k:  s_k(l) = sum_{j<k} l^j = (1 - l^k) / (1 - l)     (Eq. series; telescoping,
          Sec. 2.2, applied to scalars)
  * the general radix iteration after levels f_1..f_t (Sec. 5.3): by Lemma 5.7
          Y_t = (I - A)^{-1} (I - R_t),  R_t = E_t(...E_1(A)),
          E_i(z) = 1 - (1 - z) f_i(z)                       (Def. 5.2)
    hence y_t(l) = (1 - E_t(...E_1(l))) / (1 - l).

Q is applied reflector by reflector, O(r n^2), never formed. On probe vectors,
horner_probes_factored applies A = Q diag(lam) Q^T + X Y^T from those factors.
"""

from __future__ import annotations

import numpy as np

from .circuits import scalar_algebra


def symmetric_function(V, lam, fvals):
    """Q diag(fvals) Q^T with Q = H_1 ... H_r (rows of V are the v_i)."""
    r = V.shape[0]
    M = np.diag(np.asarray(fvals, dtype=np.float64))
    # Q M Q^T = H_1 ... H_r M H_r ... H_1 ; M stays symmetric at every step
    for i in reversed(range(r)):
        v = V[i]
        beta = 2.0 / float(v @ v)
        w = v @ M
        M = M - np.outer(beta * v, w)
        u = M @ v
        M = M - np.outer(beta * u, v)
    return M


def symmetric_function_rows(V, lam, fvals, rows):
    """Selected rows of Q diag(fvals) Q^T: row_i = Q diag(f) Q^T e_i (symmetric)."""
    r = V.shape[0]
    E = np.zeros((V.shape[1], len(rows)))
    E[np.asarray(rows), np.arange(len(rows))] = 1.0
    W = E
    for i in range(r):  # Q^T e_i = H_r ... H_1 e_i: apply H_1 first
        v = V[i]
        W = W - np.outer((2.0 / float(v @ v)) * v, v @ W)
    W = np.asarray(fvals)[:, None] * W
    for i in reversed(range(r)):  # Q u = H_1 ... H_r u: apply H_r first
        v = V[i]
        W = W - np.outer((2.0 / float(v @ v)) * v, v @ W)
    return W.T


def sk_scalar(lam, k: int):
    """s_k(l) = (1 - l^k) / (1 - l) for |l| < 1."""
    lam = np.asarray(lam, dtype=np.float64)
    return (1.0 - lam ** k) / (1.0 - lam)


def error_map(f):
    """E(z) = 1 - (1 - z) f(z) (Def. 5.2) for a kernel circuit f, on scalar arrays."""

    def E(z):
        z = np.asarray(z, dtype=np.float64)
        alg = scalar_algebra(z.shape)
        return 1.0 - (1.0 - z) * f(z, alg)

    return E


def radix_scalar(lam, levels, kernels):
    """y_t(l) = (1 - E_t(...E_1(l))) / (1 - l) (Lemma 5.7) for the given level radices."""
    lam = np.asarray(lam, dtype=np.float64)
    z = lam
    for m in levels:
        z = error_map(kernels[m])(z)
    return (1.0 - z) / (1.0 - lam)


def horner_probes(A, X, k: int):
    """S_k(A) X by s <- x + A s, k - 1 times (the definition, Eq. neumann, on vectors)."""
    S = X.copy()
    for _ in range(k - 1):
        S = X + A @ S
    return S


def horner_probes_factored(V, lam, X, Y, P, k: int):
    """S_k(A) P by the same recursion s <- p + A s (k - 1 times), with A applied
    from the factors its generator built it from: A = Q diag(lam) Q^T + X Y^T,
    Q = H_1 ... H_r, H_i = I - b_i v_i v_i^T (rows of V are the v_i).

    Q in compact WY form: Q = I - U T U^T with U = [v_1 .. v_r] and T upper
    triangular, built one reflector at a time from
      (I - U T U^T)(I - b v v^T) = I - [U v] [[T, -b T U^T v], [0, b]] [U v]^T.
    With D = diag(lam) and Z = [U, D U],
      Q D Q^T = D - U T (D U)^T - (D U) T^T U^T + U (T (U^T D U) T^T) U^T
              = D + Z C Z^T,  C = [[T G T^T, -T], [-T^T, 0]],  G = U^T D U,
    so A s = lam * s + [Z C, X] ([Z, Y]^T s): O(n (2r + rank) p) per product
    instead of O(n^2 p), which makes the definition affordable at n = 16384
    (3374 steps on 64 probes) on the host."""
    V = np.asarray(V, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    r = V.shape[0]
    U = V.T.copy()
    T = np.zeros((r, r))
    for j in range(r):
        b = 2.0 / float(V[j] @ V[j])
        T[j, j] = b
        if j:
            T[:j, j] = -b * (T[:j, :j] @ (U[:, :j].T @ V[j]))
    DU = lam[:, None] * U
    G = U.T @ DU
    C = np.block([[T @ G @ T.T, -T], [-T.T, np.zeros((r, r))]])
    Z = np.hstack([U, DU])
    left = np.hstack([Z @ C, X])
    right = np.hstack([Z, Y])
    S = np.array(P, dtype=np.float64, copy=True)
    for _ in range(k - 1):
        S = P + lam[:, None] * S + left @ (right.T @ S)
    return S


def rel_fro(X, Xref) -> float:
    """||X - Xref||_F / ||Xref||_F."""
    X = np.asarray(X, dtype=np.float64)
    Xref = np.asarray(Xref, dtype=np.float64)
    return float(np.linalg.norm(X - Xref) / np.linalg.norm(Xref))
