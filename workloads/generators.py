"""Seeded input generators (random matrices only, no series arithmetic).

Every generator is deterministic in its seed. Sub-streams come from
``numpy.random.SeedSequence(seed).spawn`` so that, for example, the eigenvalues
of a planted spectrum do not change when the number of reflectors does.

The matrix models follow the paper's experimental setup (Sec. 6, "Setup":
A = alpha * Omega D Omega^T with Omega orthogonal and D diagonal in [-1, 1]),
with Omega realised as a product of Householder reflectors so that A can be
formed in O(n^2) per reflector at n up to 16384.
"""

from __future__ import annotations

from fractions import Fraction

import numpy as np

#: Bumped whenever any generator's output for a given seed changes.
GEN_VERSION = 1


def _rngs(seed: int, count: int):
    return [np.random.default_rng(s) for s in np.random.SeedSequence(seed).spawn(count)]


def gaussian_scaled(n: int, norm2: float = 0.5, seed: int = 1000) -> dict:
    """Nonsymmetric A = norm2 * G / ||G||_2 with G i.i.d. N(0, 1).

    ||A||_2 = norm2, hence rho(A) <= norm2 < 1.
    """
    (rg,) = _rngs(seed, 1)
    G = rg.standard_normal((n, n))
    s = np.linalg.norm(G, 2) if n > 0 else 1.0
    A = (norm2 / s) * G
    return {"kind": "gaussian", "n": n, "A": A, "norm2": norm2, "seed": seed}


def _apply_reflector_both_sides(M: np.ndarray, v: np.ndarray, block: int = 2048) -> None:
    """M <- H M H in place, H = I - 2 v v^T / (v^T v) (symmetric, orthogonal)."""
    beta = 2.0 / float(v @ v)
    # H M = M - beta v (v^T M)
    w = v @ M
    n = M.shape[0]
    for r0 in range(0, n, block):
        M[r0:r0 + block] -= np.outer(beta * v[r0:r0 + block], w)
    # (H M) H = HM - beta (HM v) v^T
    u = M @ v
    for r0 in range(0, n, block):
        M[r0:r0 + block] -= np.outer(beta * u[r0:r0 + block], v)


def planted_symmetric(n: int, rho: float, seed: int, n_reflectors: int = 8) -> dict:
    """Symmetric A = Q diag(lam) Q^T, lam ~ U[-rho, rho], Q = H_1 ... H_r.

    Returns the reflector vectors V (r x n, H_i uses V[i]) and lam so that a
    closed form in the eigenbasis can be formed by whoever needs one.
    """
    rv, rl = _rngs(seed, 2)
    V = rv.standard_normal((n_reflectors, n))
    lam = rl.uniform(-rho, rho, n)
    M = np.diag(lam)
    # Q M Q^T = H_1 (H_2 ( ... (H_r M H_r) ... ) H_2) H_1
    for i in reversed(range(n_reflectors)):
        _apply_reflector_both_sides(M, V[i])
    M = 0.5 * (M + M.T)
    return {"kind": "planted", "n": n, "A": M, "V": V, "lam": lam, "rho": rho, "seed": seed}


def planted_spectrum(lam: np.ndarray, seed: int, n_reflectors: int = 8) -> dict:
    """Symmetric A = Q diag(lam) Q^T for given eigenvalues, Q = H_1 ... H_r
    (the construction of planted_symmetric with a prescribed spectrum)."""
    lam = np.asarray(lam, dtype=np.float64)
    n = lam.shape[0]
    (rv,) = _rngs(seed, 1)
    V = rv.standard_normal((n_reflectors, n))
    M = np.diag(lam)
    for i in reversed(range(n_reflectors)):
        _apply_reflector_both_sides(M, V[i])
    M = 0.5 * (M + M.T)
    return {"kind": "planted", "n": n, "A": M, "V": V, "lam": lam, "seed": seed}


def convergence_spd(d: int = 64, kappa: float = 1e4, seed: int = 6400) -> dict:
    """The convergence problem of the numerical validation: I - A symmetric
    positive definite with eigenvalues geometrically spaced in [1/kappa, 1]
    (condition number kappa), i.e. A with eigenvalues 1 - sigma_i,
    sigma_i = kappa^(-i/(d-1)), so rho(A) = 1 - 1/kappa."""
    sigma = kappa ** (-np.arange(d) / (d - 1))
    out = planted_spectrum(1.0 - sigma, seed)
    out["kappa"] = kappa
    return out


def planted_perturbed(n: int, rho: float, seed: int, rank: int = 32, pert_norm: float = 0.01,
                      n_probes: int = 64, n_reflectors: int = 8) -> dict:
    """Planted symmetric spectrum plus a nonsymmetric rank-`rank` term of 2-norm `pert_norm`.

    Delta = X Y^T with X, Y i.i.d. N(0, 1) (n x rank), scaled so ||Delta||_2 = pert_norm.
    Also returns `n_probes` N(0, 1) probe vectors (n x n_probes).
    """
    base = planted_symmetric(n, rho, seed, n_reflectors)
    rx, rp = _rngs(seed + 7_000_000, 2)
    X = rx.standard_normal((n, rank))
    Y = rx.standard_normal((n, rank))
    _, Rx = np.linalg.qr(X)
    _, Ry = np.linalg.qr(Y)
    s = np.linalg.norm(Rx @ Ry.T, 2)
    X *= pert_norm / s
    A = base["A"] + X @ Y.T
    probes = rp.standard_normal((n, n_probes))
    out = dict(base)
    out.update({"kind": "planted_perturbed", "A": A, "X": X, "Y": Y, "probes": probes,
                "pert_norm": pert_norm})
    return out


def jacobi_batch(count: int, seed: int, sizes=tuple(range(16, 257, 16)), damped: bool = True) -> list:
    """Jacobi iteration matrices of SPD systems G = H^T H + 0.1 I, H ~ N(0,1) (2n x n).

    Undamped: A = I - D^{-1} G (rho(A) > 1 for these G, kept for failure tests).
    Damped:   A = I - omega D^{-1} G, omega = 2 / (lmin + lmax) of D^{-1/2} G D^{-1/2},
              which puts the spectrum of A in [-(lmax-lmin)/(lmax+lmin), +same].
    """
    rs, rh = _rngs(seed, 2)
    ns = rs.choice(np.asarray(sizes), size=count)
    out = []
    for i in range(count):
        n = int(ns[i])
        (r,) = _rngs(int(rh.integers(0, 2**62)), 1)
        H = r.standard_normal((2 * n, n))
        G = H.T @ H + 0.1 * np.eye(n)
        d = np.diag(G).copy()
        if damped:
            sd = 1.0 / np.sqrt(d)
            ev = np.linalg.eigvalsh(G * sd[:, None] * sd[None, :])
            omega = 2.0 / (ev[0] + ev[-1])
        else:
            omega = 1.0
        A = np.eye(n) - omega * (G / d[:, None])
        out.append({"kind": "jacobi", "n": n, "A": A, "omega": omega})
    return out


def nonnormal_triangular(n: int, rho: float, seed: int, offdiag_scale: float = 1.0) -> dict:
    """Upper-triangular A with eigenvalues (its diagonal) ~ U[-rho, rho] and
    N(0, offdiag_scale^2 / n) strictly-upper entries (Sec. 6, nonnormal test)."""
    rl, ru = _rngs(seed, 2)
    lam = rl.uniform(-rho, rho, n)
    A = np.triu(ru.standard_normal((n, n)) * (offdiag_scale / np.sqrt(max(n, 1))), 1)
    A[np.diag_indices(n)] = lam
    return {"kind": "nonnormal", "n": n, "A": A, "lam": lam, "seed": seed}


def rational_small(n: int, seed: int) -> list:
    """Small matrix of exact rationals p/q, |p| <= 3, 4 <= q <= 9, scaled by 1/n."""
    (r,) = _rngs(seed, 1)
    return [[Fraction(int(r.integers(-3, 4)), int(r.integers(4, 10)) * n) for _ in range(n)]
            for _ in range(n)]


# The five workloads the library is measured on. `r` selects an independent repeat.
CONFIGS = {
    1: "gaussian n=256 ||A||_2=0.5 (k=81)",
    2: "planted symmetric n=4096 lam~U[-0.9,0.9] (k=729 radix 9, k=225 radix 15)",
    3: "planted symmetric n=8192 lam~U[-0.97,0.97] (k=3375 radix 15, k=6561 radix 9)",
    4: "4096 damped-Jacobi matrices n in {16..256} (k=81, k=225)",
    5: "planted n=16384 lam~U[-0.95,0.95] + rank-32 perturbation ||.||_2=0.01, 64 probes (k=3375)",
}


def config_inputs(cfg: int, r: int = 0, n: int | None = None, count: int | None = None) -> dict:
    """Inputs of workload `cfg` (1..5), repeat `r`, seed 1000*cfg + r.

    `n` (cfg 1, 2, 3, 5) or `count` (cfg 4) shrink a workload for tests while
    keeping its construction.
    """
    seed = 1000 * cfg + r
    if cfg == 1:
        return gaussian_scaled(n or 256, 0.5, seed)
    if cfg == 2:
        return planted_symmetric(n or 4096, 0.9, seed)
    if cfg == 3:
        return planted_symmetric(n or 8192, 0.97, seed)
    if cfg == 4:
        return {"kind": "batch", "mats": jacobi_batch(count or 4096, seed)}
    if cfg == 5:
        return planted_perturbed(n or 16384, 0.95, seed)
    raise ValueError(f"unknown workload {cfg}")
